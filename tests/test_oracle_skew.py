"""Pins of the oracle's contribution-skew statistic (Sec. 1 "Rendering
Inefficiency", Sec. 3.4 "Motivation": per pixel, the share of Gaussians whose
largest contributions Gamma alpha make up 99% of the pixel) against facts
fixed outside of it (CPU only): a brute-force walk of all visible Gaussians in
depth order, the closed form for a stack of identical Gaussians, and the
invariants of a sorted prefix."""
import math

import numpy as np

import oracle
from tests.scene_helpers import camera, scene


def _tiny(seed=0, n=60, W=40, H=30):
    rs = np.random.default_rng(seed)
    cam = camera(f=36.0, width=W, height=H)
    s = scene(rs.uniform(-0.6, 0.6, (n, 3)) + [0, 0, 4], log_scales=rs.normal(math.log(0.12), 0.3, (n, 3)),
              quats=rs.standard_normal((n, 4)), opacity=rs.uniform(0.1, 0.95, n), dc=rs.uniform(-1, 1, (n, 3)))
    return s, cam


def test_skew_matches_a_brute_force_walk():
    s, cam = _tiny()
    opts = oracle.Options()
    s64 = oracle.Scene64.from_scene(s)
    r, proj, tile, gid, ranges = oracle.render(s64, cam, opts)
    sk = oracle.contribution_skew(proj, gid, ranges, cam, opts, 0.99)
    vis = np.nonzero(proj["visible"])[0]
    order = vis[np.lexsort((vis, proj["depth32"][vis].view(np.uint32)))]
    tx_n, _ = oracle.tile_grid(cam, opts)
    checked = 0
    for y in range(cam["height"]):
        for x in range(0, cam["width"], 2):
            T, contrib, stop = 1.0, [], None
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
                    stop = g
                    break
                contrib.append(T * al)
                T *= 1 - al
            w = np.sort(np.array(contrib))[::-1]
            total = w.sum()
            m = int(np.searchsorted(np.cumsum(w), 0.99 * total) + 1) if w.size else 0
            assert sk["blended"][y, x] == len(contrib)
            assert sk["m"][y, x] == m, (x, y)
            np.testing.assert_allclose(sk["total"][y, x], total, rtol=1e-12, atol=0)
            np.testing.assert_allclose(sk["total"][y, x], 1.0 - r.T[y, x], rtol=1e-12, atol=1e-15)
            # walked: the tile's whole list, or up to the Gaussian that stopped it
            t = (y // opts.tile_h) * tx_n + x // opts.tile_w
            lst = gid[ranges[t, 0]:ranges[t, 1]]
            if stop is None:
                assert sk["walked"][y, x] == lst.size
            else:
                assert lst[sk["walked"][y, x] - 1] == stop
            checked += 1
    assert checked > 500 and sk["m"].max() > 1


def test_skew_of_a_stack_of_identical_gaussians_has_the_closed_form():
    """n identical Gaussians one behind the other: at the centre pixel every
    alpha is the same a, the contributions a (1 - a)^(i - 1) are already in
    descending order, and the m largest sum to 1 - (1 - a)^m."""
    n = 10
    means = np.array([[0.0, 0.0, 4.0 + 0.01 * i] for i in range(n)])
    W = H = 32
    cam = camera(f=40.0, width=W, height=H)
    cam["cx"] = cam["cy"] = 16.5  # the centre pixel sits on the means
    s = scene(means, log_scales=np.full((n, 3), math.log(0.2)), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
              opacity=np.full(n, 0.5), dc=np.zeros((n, 3)))
    opts = oracle.Options()
    r, proj, tile, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, opts)
    a = 0.5
    for frac in (0.5, 0.9, 0.99, 0.999):
        sk = oracle.contribution_skew(proj, gid, ranges, cam, opts, frac)
        total = 1.0 - (1.0 - a) ** n
        m = math.ceil(math.log(1.0 - frac * total) / math.log(1.0 - a))
        assert sk["blended"][16, 16] == n
        assert sk["m"][16, 16] == m, (frac, sk["m"][16, 16], m)
        np.testing.assert_allclose(sk["total"][16, 16], total, rtol=1e-12)


def test_skew_invariants():
    s, cam = _tiny(seed=3, n=120, W=48, H=40)
    opts = oracle.Options()
    r, proj, tile, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, opts)
    prev = None
    for frac in (1e-9, 0.5, 0.9, 0.99, 1.0):
        sk = oracle.contribution_skew(proj, gid, ranges, cam, opts, frac)
        b, m = sk["blended"], sk["m"]
        assert np.all(m <= b) and np.all(b <= sk["walked"])
        assert np.array_equal(m == 0, b == 0)
        if frac == 1e-9:
            assert np.all(m[b > 0] == 1)
        if frac == 1.0:
            assert np.array_equal(m, b)
        if prev is not None:
            assert np.all(m >= prev)
        prev = m
    assert (b > 0).sum() > 200 and b.max() > 20
