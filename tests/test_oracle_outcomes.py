"""Pins of the oracle's near-threshold outcome enumeration (CPU only).

``oracle.pixel_outcomes`` lists, per pixel, every result the FP64 render can
reach when decisions taken close to their thresholds go the other way (the
decision-aware comparison with an FP32 render).  It is pinned by closed forms
on hand-built scenes (a flipped support test, a flipped stop rule, a flipped
leader test of Alg. 1), by the ordinary render (outcome 0, and the only one
at tolerance 0), and by renders of slightly perturbed conics, an independent
way of making near decisions flip: every perturbed pixel must be one of the
enumerated outcomes.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from tests.scene_helpers import camera, scene

AT = 1.0 / 255.0
C0 = 0.5 / math.sqrt(math.pi)  # real SH basis Y_00 = 1 / (2 sqrt(pi))


def _setup(s, cam, opts):
    r, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, opts, 4)
    return r, proj, gid, ranges


def _outcomes(proj, gid, ranges, cam, opts, x, y, tol=1e-3):
    out, n = oracle.pixel_outcomes(proj, gid, ranges, cam, opts, [y * int(cam["width"]) + x], tol=tol)
    assert n[0] > 0
    return out[0, :n[0]]


def _sigma2(f, s, Z):
    return (f * s / Z) ** 2 + 0.3


@pytest.mark.parametrize("inside", [True, False])
def test_support_flip_closed_form(inside):
    """One isotropic Gaussian on the axis, sized so that a pixel lies at
    q = 9 (1 -+ 4e-4) from its centre: the render blends it or not (closed
    form alpha = o exp(-q/2)), and the enumeration holds both results."""
    f, Z, W = 100.0, 5.0, 64
    cam = camera(f=f, width=W, height=W, cx=W / 2 + 0.5, cy=W / 2 + 0.5)
    x, y = W // 2 + 7, W // 2            # 7 px right of the centre pixel
    q_target = 9.0 * (1 - 4e-4 if inside else 1 + 4e-4)
    sig2 = 49.0 / q_target
    s_world = math.sqrt(sig2 - 0.3) * Z / f
    o, c = 0.7, 0.8
    sc = scene([[0, 0, Z]], log_scales=[math.log(s_world)] * 3, opacity=o, dc=(c - 0.5) / C0)
    opts = oracle.Options()
    r, proj, gid, ranges = _setup(sc, cam, opts)
    np.testing.assert_allclose(proj["cov2"][0][[0, 2]], sig2, rtol=1e-12)
    al = o * math.exp(-0.5 * q_target)
    blended = np.array([al * c, al * c, al * c, 1 - al])
    empty = np.array([0.0, 0.0, 0.0, 1.0])
    outs = _outcomes(proj, gid, ranges, cam, opts, x, y)
    assert outs.shape[0] == 2
    first, second = (blended, empty) if inside else (empty, blended)
    np.testing.assert_allclose(outs[0], first, atol=1e-12)
    np.testing.assert_allclose(outs[1], second, atol=1e-12)
    # outcome 0 is the render's pixel
    np.testing.assert_allclose(outs[0][:3], r.rgb[:, y, x], atol=0)
    # far from the boundary there is one outcome
    assert _outcomes(proj, gid, ranges, cam, opts, W // 2, W // 2).shape[0] == 1


@pytest.mark.parametrize("above", [True, False])
def test_stop_rule_flip_closed_form(above):
    """Five identical Gaussians hit at their centres with 1 - o chosen so that
    T after four blends is Gamma_theta (1 +- 2e-4): the pixel stops before or
    after the fourth, and the enumeration holds both closed forms."""
    W = 64
    cam = camera(f=100.0, width=W, height=W, cx=W / 2 + 0.5, cy=W / 2 + 0.5)
    t4 = 1e-4 * (1 + 2e-4 if above else 1 - 2e-4)
    o = 1 - t4 ** 0.25
    c = 0.6
    sc = scene([[0, 0, z] for z in (2, 3, 4, 5, 6)], log_scales=[math.log(0.2)] * 3, opacity=o,
               dc=(c - 0.5) / C0)
    opts = oracle.Options()
    r, proj, gid, ranges = _setup(sc, cam, opts)

    def after(j):  # state after j blends
        T = (1 - o) ** j
        return np.array([c * (1 - T)] * 3 + [T])

    outs = _outcomes(proj, gid, ranges, cam, opts, W // 2, W // 2)
    assert outs.shape[0] == 2
    first, second = (after(4), after(3)) if above else (after(3), after(4))
    np.testing.assert_allclose(outs[0], first, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(outs[1], second, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(outs[0][3], r.T[W // 2, W // 2], rtol=1e-14)


def test_leader_flip_closed_form():
    """Alg. 1 with 2x2 groups: a Gaussian whose support edge passes within
    4e-4 of the group leader while the pixel diagonal to it is well inside.
    The leader test may flip, so that pixel may receive the Gaussian or not."""
    f, Z, W = 100.0, 5.0, 64
    lx, ly = 32, 32                       # a group leader (even coordinates)
    sig2 = 2.0
    q_lead = 9.0 * (1 - 4e-4)
    # the Gaussian on the optical axis (isotropic Sigma'), the principal point
    # on the diagonal through the leader, towards the group's far pixel
    d = math.sqrt(q_lead * sig2 / 2)
    u = lx + 0.5 + d
    cam = camera(f=f, width=W, height=W, cx=u, cy=u)
    s_world = math.sqrt(sig2 - 0.3) * Z / f
    o, c = 0.9, 0.7
    sc = scene([[0, 0, Z]], log_scales=[math.log(s_world)] * 3, opacity=o, dc=(c - 0.5) / C0)
    opts = oracle.Options(cr=True, group_w=2, group_h=2)
    r, proj, gid, ranges = _setup(sc, cam, opts)
    np.testing.assert_allclose(proj["uv"][0], [u, u], rtol=1e-12)
    # the pixel (lx + 1, ly + 1): q there, closed form
    qp = 2 * (u - (lx + 1.5)) ** 2 / sig2
    al = o * math.exp(-0.5 * qp)
    assert qp < 8 and al > 10 * AT
    outs = _outcomes(proj, gid, ranges, cam, opts, lx + 1, ly + 1)
    assert outs.shape[0] == 2
    np.testing.assert_allclose(outs[0], [al * c] * 3 + [1 - al], atol=1e-12)   # leader passes (FP64)
    np.testing.assert_allclose(outs[1], [0, 0, 0, 1], atol=1e-12)              # the group skips it
    # the plain rule has no leader: one outcome
    plain = oracle.Options()
    rp, projp, gidp, rangesp = _setup(sc, cam, plain)
    assert _outcomes(projp, gidp, rangesp, cam, plain, lx + 1, ly + 1).shape[0] == 1


def _scene_10k(W=256, H=224):
    sc, cams = scenegen.uniform_10k(width=W, height=H)
    cam = cams[0]
    cam["fx"] = cam["fy"] = 220.0
    return sc, cam


OPTS = {
    "plain": oracle.Options(),
    "cr2x2": oracle.Options(cr=True, group_w=2, group_h=2),
    "cr2x4_opacity": oracle.Options(cr=True, group_w=2, group_h=4, opacity_filter=True),
}


@pytest.mark.parametrize("name", sorted(OPTS))
def test_outcome_zero_is_the_render(name):
    sc, cam = _scene_10k()
    opts = OPTS[name]
    r, proj, gid, ranges = _setup(sc, cam, opts)
    W, H = cam["width"], cam["height"]
    pix = np.arange(W * H)
    out, n = oracle.pixel_outcomes(proj, gid, ranges, cam, opts, pix, tol=1e-3, nthreads=4)
    assert (n >= 1).all()
    assert np.array_equal(out[:, 0, :3], r.rgb.reshape(3, -1).T)
    assert np.array_equal(out[:, 0, 3], r.T.reshape(-1))
    # pixels whose decisions are all clear of their thresholds have one outcome
    clear = r.margin.reshape(-1) >= 1e-3
    assert (n[clear] == 1).all()
    assert (n[~clear] >= 2).sum() > 0
    # at tolerance 0 nothing branches
    out0, n0 = oracle.pixel_outcomes(proj, gid, ranges, cam, opts, pix, tol=0.0, max_out=1, nthreads=4)
    assert (n0 == 1).all() and np.array_equal(out0[:, 0], out[:, 0])
    # every outcome is a valid composite: 0 <= T <= 1, colour within [0, max colour]
    for k in range(out.shape[1]):
        m = n > k
        assert ((out[m, k, 3] >= 0) & (out[m, k, 3] <= 1)).all()
        assert (out[m, k, :3] >= -1e-15).all()


@pytest.mark.parametrize("name", sorted(OPTS))
@pytest.mark.parametrize("delta", [1e-4, -1e-4])
def test_perturbed_renders_are_enumerated_outcomes(name, delta):
    """Scaling every conic by 1 + delta moves q by a relative delta, which
    flips decisions near their thresholds (support, alpha, stop, leader) the
    way single-precision rounding can.  Each pixel of the perturbed render must
    equal, within the perturbation's continuous effect, one of the outcomes
    enumerated on the unperturbed scene at tolerance 1e-3 -- and some pixels
    must match only a flipped outcome."""
    sc, cam = _scene_10k()
    opts = OPTS[name]
    r, proj, gid, ranges = _setup(sc, cam, opts)
    pert = proj.copy()
    pert["conic"] *= 1 + delta
    rp = oracle.render_tiled(pert, gid, ranges, cam, opts, 4)
    W, H = cam["width"], cam["height"]
    pix = np.arange(W * H)
    out, n = oracle.pixel_outcomes(proj, gid, ranges, cam, opts, pix, tol=1e-3, nthreads=4)
    assert (n > 0).all()
    val = np.concatenate([rp.rgb.reshape(3, -1).T, rp.T.reshape(-1, 1)], 1)
    err = np.abs(out - val[:, None, :]).max(2)
    err[np.arange(out.shape[1])[None, :] >= n[:, None]] = np.inf
    # continuous effect of the perturbation: |d alpha| <= alpha q |delta| / 2 per layer
    best = err.min(1)
    assert best.max() <= 2e-4, best.max()
    flipped_only = (err[:, 0] > 2e-4) & (best <= 2e-4)
    assert flipped_only.sum() >= 5, flipped_only.sum()
