"""Pins of the FP64 oracle against facts fixed outside of it (CPU only).

Each test checks the oracle against a closed form, a library routine, a brute
force computation or an invariant the paper's equations imply, chosen so that
a plausible slip (a dropped term, a transposed operand, a sign) fails one.
"""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy.spatial.transform import Rotation

import oracle
import scenegen
from tests.scene_helpers import camera, scene

AT = 1.0 / 255.0


def _render(s, cam, opts=None, nthreads=4):
    opts = opts or oracle.Options()
    r, proj, tile, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, opts, nthreads)
    return r, proj


def _y00():
    return sps.sph_harm_y(0, 0, 0.0, 0.0).real


# ----------------------------------------------------------- projection --

@pytest.mark.parametrize("log_s,opacity", [(math.log(0.1), 0.9), (math.log(0.5), 0.995)])
def test_single_isotropic_gaussian_on_axis_closed_form(log_s, opacity):
    """Eqn. 2 for one isotropic Gaussian on the optical axis: Sigma' is
    ((f s / Z)^2 + 0.3) I, so alpha(p) = min(.99, o exp(-|p - c|^2 / (2 sigma^2)))."""
    f, Z, W = 100.0, 5.0, 64
    cam = camera(f=f, width=W, height=W)
    s = scene([[0, 0, Z]], log_scales=[log_s] * 3, opacity=opacity, dc=0.0)
    r, proj = _render(s, cam)
    sig2 = (f * math.exp(log_s) / Z) ** 2 + 0.3
    ys, xs = np.mgrid[0:W, 0:W]
    d2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - W / 2) ** 2
    q = d2 / sig2
    al = np.minimum(0.99, opacity * np.exp(-0.5 * q))
    keep = (q <= 9.0) & (al >= AT)
    exp_c = np.where(keep, 0.5 * al, 0.0)
    np.testing.assert_allclose(r.rgb[0], exp_c, atol=1e-12)
    np.testing.assert_allclose(r.T, np.where(keep, 1 - al, 1.0), atol=1e-12)
    assert proj["visible"][0] == 1
    if opacity > 0.99:
        assert r.counters["clamped"] > 0


def test_ewa_covariance_matches_monte_carlo_projection():
    """EWA (Zwicker et al.) is the local affine approximation of the pinhole
    projection: sampling the 3D Gaussian and projecting each sample must give
    the oracle's Sigma' - 0.3 I and (u, v)."""
    rs = np.random.default_rng(3)
    Rc = Rotation.from_euler("xyz", [0.2, -0.3, 0.15]).as_matrix()
    tc = np.array([0.3, -0.2, 1.0])
    cam = camera(f=800.0, width=1280, height=720, cx=640.0, cy=360.0, R=Rc, t=tc)
    centre_cam = np.array([1.1, -0.7, 12.0])
    mean = Rc.T @ (centre_cam - tc)
    q_xyzw = Rotation.random(random_state=5).as_quat()
    quat_wxyz = np.array([q_xyzw[3], q_xyzw[0], q_xyzw[1], q_xyzw[2]])
    scales = np.array([0.02, 0.006, 0.012])
    s = scene([mean], log_scales=np.log(scales), quats=[quat_wxyz])
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, oracle.Options())
    assert proj["visible"][0] == 1
    Rg = Rotation.from_quat(q_xyzw).as_matrix()
    N = 1_000_000
    pts = mean + (rs.standard_normal((N, 3)) * scales) @ Rg.T
    pc = pts @ Rc.T + tc
    uv = np.stack([cam["fx"] * pc[:, 0] / pc[:, 2] + cam["cx"], cam["fy"] * pc[:, 1] / pc[:, 2] + cam["cy"]], 1)
    cov_mc = np.cov(uv.T)
    a, b, c = proj["cov2"][0]
    cov_or = np.array([[a - 0.3, b], [b, c - 0.3]])
    assert np.linalg.norm(cov_mc - cov_or) / np.linalg.norm(cov_or) < 0.01
    np.testing.assert_allclose(uv.mean(0), proj["uv"][0], atol=0.02)
    # the conic is the inverse of Sigma'
    A, B, C = proj["conic"][0]
    np.testing.assert_allclose(np.array([[A, B], [B, C]]) @ np.array([[a, b], [b, c]]), np.eye(2), atol=1e-12)


def test_quaternion_rotates_long_axis():
    """q = (cos 22.5, 0, 0, sin 22.5) turns the x axis by +45 deg about z, so a
    Gaussian elongated along x projects (x right, y down) with a positive
    off-diagonal; its principal axis is q e_x q* (Hamilton product)."""
    h = math.radians(22.5)
    q = np.array([math.cos(h), 0, 0, math.sin(h)])
    cam = camera(f=100.0)
    s = scene([[0, 0, 10]], log_scales=np.log([0.5, 0.05, 0.05]), quats=[q])
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, oracle.Options())
    a, b, c = proj["cov2"][0]
    assert b > 0
    w, v = np.linalg.eigh(np.array([[a, b], [b, c]]))
    axis = v[:, 1] * np.sign(v[0, 1])

    def hamilton(p, r):
        return np.array([p[0] * r[0] - p[1] * r[1] - p[2] * r[2] - p[3] * r[3],
                         p[0] * r[1] + p[1] * r[0] + p[2] * r[3] - p[3] * r[2],
                         p[0] * r[2] - p[1] * r[3] + p[2] * r[0] + p[3] * r[1],
                         p[0] * r[3] + p[1] * r[2] - p[2] * r[1] + p[3] * r[0]])
    rot_x = hamilton(hamilton(q, [0, 1, 0, 0]), q * np.array([1, -1, -1, -1]))[1:]
    np.testing.assert_allclose(axis, rot_x[:2] / np.linalg.norm(rot_x[:2]), atol=1e-9)


def test_sigma_block_matches_scipy_rotation():
    """Far on the optical axis with an identity camera, Sigma' = (f/Z)^2 Sigma[:2,:2] + 0.3 I
    where Sigma = R S^2 R^T is built here with scipy's rotation."""
    rs = np.random.default_rng(11)
    f, Z = 100.0, 50.0
    cam = camera(f=f)
    for _ in range(5):
        q_xyzw = Rotation.random(random_state=rs.integers(1 << 30)).as_quat()
        wxyz = np.array([q_xyzw[3], *q_xyzw[:3]]) * rs.uniform(0.5, 2.0)   # unnormalised on purpose
        sc = rs.uniform(0.05, 0.5, 3)
        s = scene([[0, 0, Z]], log_scales=np.log(sc), quats=[wxyz])
        proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, oracle.Options())
        R = Rotation.from_quat(q_xyzw).as_matrix()
        Sig = R @ np.diag(sc ** 2) @ R.T
        a, b, c = proj["cov2"][0]
        np.testing.assert_allclose([a, b, c], [(f / Z) ** 2 * Sig[0, 0] + 0.3, (f / Z) ** 2 * Sig[0, 1],
                                               (f / Z) ** 2 * Sig[1, 1] + 0.3], rtol=1e-12, atol=1e-12)


def test_frustum_and_near_culling():
    cam = camera(f=100.0, width=64, height=64)
    lim = 1.3 * 64 / 200.0
    s = scene([[0, 0, 0.1], [0, 0, -3], [lim * 5 * 1.01, 0, 5], [lim * 5 * 0.99, 0, 5], [0, 0, 0.3]],
              log_scales=[math.log(0.001)] * 3)
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, oracle.Options())
    # behind near, behind camera, outside 1.3x FOV: culled; the 4th is inside the
    # slack but its 1-pixel footprint is off-image, so it touches no tile either
    assert list(proj["visible"]) == [0, 0, 0, 0, 1]


# ------------------------------------------------------------------- SH --

def _real_sh_scipy(lmax, d):
    th = np.arccos(np.clip(d[:, 2], -1, 1))
    ph = np.arctan2(d[:, 1], d[:, 0])
    cols = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            Y = sps.sph_harm_y(l, abs(m), th, ph)
            cols.append(Y.real if m == 0 else math.sqrt(2) * (Y.real if m > 0 else Y.imag))
    return np.stack(cols, 1)


def test_sh_basis_matches_scipy_and_is_orthonormal():
    rs = np.random.default_rng(0)
    d = rs.standard_normal((500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y = oracle.sh_eval(3, d)
    np.testing.assert_allclose(y, _real_sh_scipy(3, d), atol=1e-13)
    # Gram matrix by product quadrature (Gauss-Legendre in cos(theta) x uniform phi)
    x, wq = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * 2 * np.pi / 32
    X, P = np.meshgrid(x, phis, indexing="ij")
    st = np.sqrt(1 - X ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), X], -1).reshape(-1, 3)
    w = (wq[:, None] * np.full(32, 2 * np.pi / 32)[None, :]).reshape(-1)
    Yq = oracle.sh_eval(3, dirs)
    np.testing.assert_allclose((Yq * w[:, None]).T @ Yq, np.eye(16), atol=1e-12)
    # 3DGS sign convention: Y_{1,-1} ~ -y, Y_{1,0} ~ z, Y_{1,1} ~ -x
    e = oracle.sh_eval(1, np.eye(3))
    assert e[1, 1] < 0 and e[2, 2] > 0 and e[0, 3] < 0


def test_sh_gradient_matches_finite_differences():
    rs = np.random.default_rng(1)
    d = rs.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    _, g = oracle.sh_eval(3, d, grad=True)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (oracle.sh_eval(3, d + e) - oracle.sh_eval(3, d - e)) / (2 * h)
        np.testing.assert_allclose(g[:, :, i], fd, atol=1e-8)


def test_colour_uses_direction_from_camera_to_gaussian():
    """Only Y_{1,0} (and then Y_{1,1}) weighted: the colour is 0.5 + k Y(d) with
    d = unit(mean - camera centre)."""
    cam = camera(f=20.0, t=[0, 0, 1.0])           # camera centre at (0, 0, -1)
    sh = np.zeros((2, 4, 3))
    sh[0, 2, :] = 0.3
    sh[1, 3, :] = -0.4
    s = scene([[0, 0, 4], [3, 0, 3]], sh=sh, sh_degree=1)
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, oracle.Options())
    assert list(proj["visible"]) == [1, 1]
    y10 = sps.sph_harm_y(1, 0, 0.0, 0.0).real
    np.testing.assert_allclose(proj["rgb_raw"][0], 0.5 + 0.3 * y10, rtol=1e-13)
    th = math.acos(0.8)
    y11 = math.sqrt(2) * sps.sph_harm_y(1, 1, th, 0.0).real
    np.testing.assert_allclose(proj["rgb_raw"][1], 0.5 - 0.4 * y11, rtol=1e-13)


# ------------------------------------------------------------- blending --

def _centre_camera(W=64):
    # pixel W/2 is sampled at W/2 + .5: put the principal point there
    return camera(f=100.0, width=W, height=W, cx=W / 2 + 0.5, cy=W / 2 + 0.5)


def test_two_gaussians_compose_with_the_over_operator():
    """Eqn. 1 for two Gaussians hit at their centres (q = 0, alpha = o):
    C = o1 c1 + (1 - o1) o2 c2 whatever their storage order."""
    cam = _centre_camera()
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.2, 0.8, 0.3])
    dc = np.stack([(c1 - 0.5) / _y00(), (c2 - 0.5) / _y00()])
    for order in ([0, 1], [1, 0]):
        s = scene(np.array([[0, 0, 4], [0, 0, 6]])[order], log_scales=[math.log(0.2)] * 3,
                  opacity=np.array([0.6, 0.7])[order], dc=dc[order])
        r, _ = _render(s, cam)
        np.testing.assert_allclose(r.rgb[:, 32, 32], 0.6 * c1 + 0.4 * 0.7 * c2, atol=1e-12)
        np.testing.assert_allclose(r.T[32, 32], 0.4 * 0.3, atol=1e-12)


def test_termination_stops_before_crossing_gamma_theta():
    """alpha = 0.95 five times: T runs 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4,
    so the fourth Gaussian is not blended and the pixel stops."""
    cam = _centre_camera()
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]], np.float64) * 0.8 + 0.1
    s = scene([[0, 0, z] for z in (2, 3, 4, 5, 6)], log_scales=[math.log(0.2)] * 3, opacity=0.95,
              dc=(cols - 0.5) / _y00())
    r, _ = _render(s, cam)
    exp = 0.95 * cols[0] + 0.05 * 0.95 * cols[1] + 0.0025 * 0.95 * cols[2]
    np.testing.assert_allclose(r.rgb[:, 32, 32], exp, atol=1e-12)
    np.testing.assert_allclose(r.T[32, 32], 1.25e-4, rtol=1e-10)
    assert r.ncontrib[32, 32] == 3


def _random_scene(n=1500, seed=2, W=100, H=70):
    sc, _ = scenegen.uniform_10k(seed=seed, n=n, width=W, height=H)
    cam = scenegen.look_at((0.3, -0.2, -3), (0, 0, 0), W, H)
    cam["fx"] = cam["fy"] = 90.0
    return sc, cam


@pytest.mark.parametrize("opts", [oracle.Options(), oracle.Options(cr=True), oracle.Options(opacity_filter=True),
                                  oracle.Options(cr=True, group_w=2, group_h=4, tile_h=16)])
def test_tiled_render_equals_bruteforce(opts):
    """Binning and per-tile sorting change nothing: every pixel equals a walk
    over all visible Gaussians in global depth order (ragged 100x70 image)."""
    s, cam = _random_scene()
    r, proj = _render(s, cam, opts)
    rgb, T = oracle.render_bruteforce(proj, cam, opts, nthreads=4)
    np.testing.assert_array_equal(r.rgb, rgb)
    np.testing.assert_array_equal(r.T, T)
    assert np.all(r.T >= opts.t_stop) and np.all(r.T <= 1.0)


@pytest.mark.parametrize("cr", [False, True])
def test_image_independent_of_tile_size(cr):
    s, cam = _random_scene()
    imgs = [_render(s, cam, oracle.Options(tile_w=tw, tile_h=th, cr=cr))[0].rgb for tw, th in ((8, 8), (16, 16), (32, 8))]
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_array_equal(imgs[0], imgs[2])


def test_opacity_aware_filter_keeps_the_image_and_drops_instances():
    """Eqns. 4-5: beyond q = 2 ln(o / alpha_theta) alpha < alpha_theta anyway,
    so the tighter support removes tile instances but no contribution."""
    s, cam = _random_scene(n=3000)
    r0, p0 = _render(s, cam)
    r1, p1 = _render(s, cam, oracle.Options(opacity_filter=True))
    np.testing.assert_array_equal(r0.rgb, r1.rgb)
    assert r1.counters["instances"] < r0.counters["instances"]
    o = p1["opacity"][p1["visible"] == 1]
    assert np.all(o > AT)
    np.testing.assert_allclose(p1["tg"][p1["visible"] == 1], np.minimum(2 * np.log(o / AT), 9.0), rtol=1e-15)


def test_ellipse_tile_test_keeps_the_image_and_is_a_subset_of_the_rect():
    """The ellipse tile test (Sec. 3.3's online filtering, tightened from the
    bounding rect to the support ellipse) drops tile instances but no pixel
    that the support q <= t_g reaches, so the image is the same."""
    s, cam = _random_scene(n=3000)
    for of in (False, True):
        rr, pr, tr, gr, _ = oracle.render(oracle.Scene64.from_scene(s), cam,
                                          oracle.Options(opacity_filter=of, tile_test="rect"), 4)
        re, pe, te, ge, _ = oracle.render(oracle.Scene64.from_scene(s), cam,
                                          oracle.Options(opacity_filter=of), 4)
        np.testing.assert_array_equal(rr.rgb, re.rgb)
        np.testing.assert_array_equal(rr.T, re.T)
        assert re.counters["alpha_evals"] < rr.counters["alpha_evals"]
        rect_set = set(zip(tr.tolist(), gr.tolist()))
        ell_set = set(zip(te.tolist(), ge.tolist()))
        assert ell_set < rect_set and len(ell_set) < 0.8 * len(rect_set)
        np.testing.assert_array_equal(pr["rect"], pe["rect"])
        assert np.all(pe["ntiles"] <= pr["ntiles"])


def _min_q_on_box(A, B, C, x0, x1, y0, y1):
    """Minimum of q = A x^2 + 2 B x y + C y^2 over the box [x0,x1] x [y0,y1]:
    zero if the box holds the origin, else the smallest of the four edge
    minima (each a 1-D quadratic minimised in closed form and clamped)."""
    if x0 <= 0 <= x1 and y0 <= 0 <= y1:
        return 0.0
    best = np.inf
    for y in (y0, y1):  # horizontal edges: q(x) = A x^2 + 2 B y x + C y^2
        x = min(max(-B * y / A, x0), x1)
        best = min(best, A * x * x + 2 * B * x * y + C * y * y)
    for x in (x0, x1):
        y = min(max(-B * x / C, y0), y1)
        best = min(best, A * x * x + 2 * B * x * y + C * y * y)
    return best


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_ellipse_tile_test_brute_force(tile):
    """A tile of the rect is kept exactly when the inflated support ellipse
    q <= t_g (1 + 1e-3) meets the rectangle of its pixel centres widened by
    1/256 px (minimum of q over that box by edge minimisation, an independent
    construction), and so every tile holding a pixel centre with q <= t_g is
    kept (checked on the pixel grid)."""
    s, cam = _random_scene(n=600)
    opts = oracle.Options(tile_w=tile[0], tile_h=tile[1], opacity_filter=True)
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, opts)
    tiles, gid, _ = oracle.instances(proj, cam, opts)
    tx_n, _ = oracle.tile_grid(cam, opts)
    kept = set(zip(gid.tolist(), tiles.tolist()))
    TW, TH = tile
    n_checked = n_dropped = 0
    for g in np.flatnonzero(proj["visible"] == 1):
        P = proj[g]
        A, B, C = P["conic"]
        t = P["tg"] * (1 + 1e-3)
        u, v = P["uv"]
        x0r, y0r, x1r, y1r = P["rect"]
        for ty in range(y0r, y1r + 1):
            for tx in range(x0r, x1r + 1):
                e = 1.0 / 256
                qmin = _min_q_on_box(A, B, C, tx * TW + 0.5 - e - u, tx * TW + TW - 0.5 + e - u,
                                     ty * TH + 0.5 - e - v, ty * TH + TH - 0.5 + e - v)
                if abs(qmin - t) < 1e-9 * t:
                    continue
                want = qmin <= t
                assert ((g, ty * tx_n + tx) in kept) == want, (g, tx, ty, qmin, t)
                xs = tx * TW + 0.5 + np.arange(TW) - u
                ys = ty * TH + 0.5 + np.arange(TH) - v
                X, Y = np.meshgrid(xs, ys)
                if np.min(A * X * X + 2 * B * X * Y + C * Y * Y) <= P["tg"]:
                    assert want
                n_checked += 1
                n_dropped += not want
    assert n_checked > 1000 and n_dropped > 0.2 * n_checked


# ------------------------------------------------------------------- CR --

def test_cr_with_one_pixel_groups_is_plain():
    s, cam = _random_scene()
    r0, _ = _render(s, cam)
    r1, _ = _render(s, cam, oracle.Options(cr=True, group_w=1, group_h=1))
    np.testing.assert_array_equal(r0.rgb, r1.rgb)
    np.testing.assert_array_equal(r0.T, r1.T)


def test_cr_equals_plain_when_every_leader_passes():
    """Large opaque Gaussians give every leader alpha >= alpha_theta, so Alg. 1
    skips nothing and matches plain blending exactly."""
    cam = camera(f=100.0, width=48, height=32)
    rs = np.random.default_rng(4)
    s = scene(rs.uniform(-0.2, 0.2, (6, 3)) + [0, 0, 6], log_scales=[math.log(2.0)] * 3,
              opacity=rs.uniform(0.05, 0.3, 6), dc=rs.uniform(-1, 1, (6, 3)))
    r0, _ = _render(s, cam)
    r1, _ = _render(s, cam, oracle.Options(cr=True))
    assert r1.counters["leader_skips"] == 0
    np.testing.assert_array_equal(r0.rgb, r1.rgb)


def test_cr_leader_decides_for_its_group():
    """Alg. 1: a Gaussian outside the leader's support is skipped by the whole
    2x2 group even where another pixel of the group would blend it; a Gaussian
    the leader keeps is blended per pixel with the alpha_theta rule (Sec. 3.4)."""
    cam = camera(f=100.0, width=64, height=64)        # pixel p sampled at p + .5
    Z = 5.0
    # centre at (31.9, 31.9): inside pixel (31, 31) of the group led by (30, 30)
    off = (31.9 - 32.0) * Z / 100.0
    s = scene([[off, off, Z]], log_scales=[math.log(1e-4)] * 3, opacity=0.9, dc=0.0)
    plain, _ = _render(s, cam)
    cr, _ = _render(s, cam, oracle.Options(cr=True))
    assert plain.rgb[0, 31, 31] > 0.1 and plain.rgb[0, 30, 30] == 0.0
    assert np.all(cr.rgb[:, 30:32, 30:32] == 0.0)
    assert cr.rgb[0, 32, 32] > 0 and cr.rgb[0, 32, 32] == plain.rgb[0, 32, 32]
    # centred on the leader (30, 30): the leader passes; pixel (31, 31) is at
    # q = 2 / 0.3 = 6.7 -> alpha = 0.9 e^-3.3 ~ 0.03 >= 1/255 so it blends too
    off = (30.5 - 32.0) * Z / 100.0
    s = scene([[off, off, Z]], log_scales=[math.log(1e-4)] * 3, opacity=0.9, dc=0.0)
    plain, _ = _render(s, cam)
    cr, _ = _render(s, cam, oracle.Options(cr=True))
    np.testing.assert_array_equal(plain.rgb[:, 30:32, 30:32], cr.rgb[:, 30:32, 30:32])
    assert cr.rgb[0, 31, 31] > 0


# ----------------------------------------------------- view clusters ------

def test_cluster_filter_equals_subset_render():
    """Sec. 3.3: rendering with the view-cluster filter is rendering the scene
    restricted to Gaussians of the selected clusters (shared ones included)."""
    sc, cams = scenegen.clusters_500k(n=20_000, width=160, height=96, n_cams=3)
    s64 = oracle.Scene64.from_scene(sc)
    for cam in cams:
        sel = oracle.select_clusters(s64.centroids, s64.pos_scale, cam, 3)
        assert bin(sel).count("1") == 4
        keep = (sc["cluster_mask"] & np.uint32(sel)) != 0
        assert 0 < keep.sum() < keep.size
        r_f, _ = _render(sc, cam, oracle.Options(use_mask=True, sel_bits=sel))
        r_s, _ = _render(scenegen.subset(sc, np.nonzero(keep)[0]), cam)
        np.testing.assert_array_equal(r_f.rgb, r_s.rgb)


def test_cluster_selection_brute_force():
    sc, cams = scenegen.clusters_500k(n=100, n_cams=8)
    cen = sc["centroids"]
    for cam in cams:
        sel = oracle.select_clusters(cen, sc["pos_scale"], cam, 3)
        R = np.asarray(cam["world_to_cam"])[:, :3]
        pos = -R.T @ np.asarray(cam["world_to_cam"])[:, 3]
        f = np.concatenate([pos / sc["pos_scale"], R[2]])
        near = int(np.argmin(((cen - f) ** 2).sum(1)))
        d = ((cen - cen[near]) ** 2).sum(1)
        order = np.argsort(d, kind="stable")
        assert order[0] == near
        assert sel == sum(1 << int(k) for k in order[:4])


# ------------------------------------------- transmittance along the list --

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_transmittance_is_monotone_along_the_list(seed):
    """Eqn. 1 composites front to back: adding the next Gaussian in depth
    order can only lower a pixel's transmittance and raise its colour (SH
    colours are clamped at 0), and the stopping rule keeps T >= Gamma_theta.
    The oracle renders the j nearest Gaussians for every j, as a black box."""
    sc, cams = scenegen.uniform_10k(seed=seed, n=40, width=24, height=24)
    # opaque, wide Gaussians, so that pixels reach Gamma_theta
    sc["opacity_logits"] = sc["opacity_logits"] + np.float32(4.0)
    sc["log_scales"] = sc["log_scales"] + np.float32(3.0)
    cam = cams[0]
    opts = oracle.Options()
    proj = oracle.preprocess(oracle.Scene64.from_scene(sc), cam, opts)
    vis = np.nonzero(proj["visible"] == 1)[0]
    order = vis[np.lexsort((vis, proj["depth32"][vis]))]
    assert order.size > 30
    prev_T = np.ones((24, 24))
    prev_C = np.zeros((3, 24, 24))
    changed = 0
    for j in range(order.size + 1):
        sub = proj.copy()
        sub["visible"] = 0
        sub["visible"][order[:j]] = 1
        C, T = oracle.render_bruteforce(sub, cam, opts)
        assert np.all(T <= prev_T) and np.all(C >= prev_C), j
        assert np.all(T >= opts.t_stop) and np.all(T <= 1.0)
        changed += int(np.any(T < prev_T))
        prev_T, prev_C = T, C
    assert changed > order.size // 2
    full = oracle.render(oracle.Scene64.from_scene(sc), cam, opts)[0]
    np.testing.assert_array_equal(full.T, prev_T)
    assert full.counters["terminated"] > 100


# ---------------------------------------------- CR error against plain ----

@pytest.mark.parametrize("group", [(2, 2), (2, 4), (4, 4)])
@pytest.mark.parametrize("seed", [3, 4])
def test_cr_differs_from_plain_by_at_most_its_skipped_alphas(seed, group):
    """Alg. 1 blends at pixel p exactly the Gaussians plain blends there
    whose test at the group's top-left pixel passes.  Removing one layer g
    from an over-composite changes it by T_front alpha_g (c_g - C_behind),
    at most alpha_g c_max per channel, and stopping at Gamma_theta leaves
    out at most T_final c_max; so per pixel and channel
        |C_plain - C_CR| <= c_max (sum of alpha_g,p over the skipped g
                                   + T_final of each run that stopped).
    The skipped set is computed here from the leader rule; the two images
    are the oracle's."""
    sc, cams = scenegen.uniform_10k(seed=seed, n=300, width=48, height=48)
    cam = cams[0]
    s64 = oracle.Scene64.from_scene(sc)
    plain = oracle.render(s64, cam, oracle.Options())[0]
    cr = oracle.render(s64, cam, oracle.Options(cr=True, group_w=group[0], group_h=group[1]))[0]
    proj = oracle.preprocess(s64, cam, oracle.Options())
    P = proj[proj["visible"] == 1]
    cmax = P["rgb"].max(axis=0)
    a_min, a_max = 1.0 / 255.0, 0.99

    def alpha_on(x, y):
        dx, dy = x - P["uv"][:, 0], y - P["uv"][:, 1]
        q = P["conic"][:, 0] * dx * dx + 2.0 * P["conic"][:, 1] * dx * dy + P["conic"][:, 2] * dy * dy
        al = np.minimum(a_max, P["opacity"] * np.exp(-0.5 * q))
        return al, (q <= P["tg"]) & (al >= a_min)

    checked = differ = 0
    for py in range(48):
        for px in range(48):
            if min(plain.margin[py, px], cr.margin[py, px]) < 1e-9:
                continue
            al, on = alpha_on(px + 0.5, py + 0.5)
            _, lead = alpha_on(px - px % group[0] + 0.5, py - py % group[1] + 0.5)
            skipped = al[on & ~lead].sum()
            stop = sum(t for t in (plain.T[py, px], cr.T[py, px]) if t < 0.01)
            d = np.abs(plain.rgb[:, py, px] - cr.rgb[:, py, px])
            assert np.all(d <= cmax * (skipped + stop) + 1e-12), (px, py, d, skipped, stop)
            if skipped == 0 and stop == 0:
                assert np.all(d == 0)   # no skip and no stop: the same layers
            checked += 1
            differ += int(np.any(d > 0))
    assert checked > 0.99 * 48 * 48 and differ > 50
