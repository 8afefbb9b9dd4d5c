"""Contribution skew on the GPU (seele_contribution_skew, Sec. 1 and Sec. 3.4
"Motivation") against the FP64 oracle: per pixel, the number m of largest
contributions Gamma alpha that make up frac of the total, the contribution
count, the tile-list entries walked and the total -- integers exact wherever
no FP32 decision or prefix cut lies within 1e-4 (relative) of a flip."""
import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _cases():
    sc, cams = scenegen.uniform_10k()
    cam2 = scenegen.look_at((0.4, -0.3, -3.2), (0, 0, 0), 100, 70)
    cam2["fx"] = cam2["fy"] = 85.0
    return sc, [cams[0], cam2]


@pytest.mark.parametrize("tile,frac", [((16, 16), 0.99), ((32, 8), 0.99), ((16, 16), 0.5)])
def test_skew_matches_oracle(Renderer, tile, frac):
    sc, cams = _cases()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    got = r.contribution_skew(frac, tile=tile)
    s64 = oracle.Scene64.from_scene(sc)
    opts = oracle.Options(tile_w=tile[0], tile_h=tile[1])
    walked_checked = 0
    for ci, cam in enumerate(cams):
        ref_r, proj, _, gid, ranges = oracle.render(s64, cam, opts, nthreads=8)
        ref = oracle.contribution_skew(proj, gid, ranges, cam, opts, frac, nthreads=8)
        g = got[ci]
        clear = ref["margin"] >= 1e-4
        assert clear.mean() > 0.8, clear.mean()
        for k in ("m", "blended"):
            bad = (g[k].astype(np.int64) != ref[k]) & clear
            assert not bad.any(), (ci, k, np.argwhere(bad)[:5])
        np.testing.assert_allclose(g["total"], ref["total"], rtol=0, atol=2e-5)
        # the entries walked and the list lengths also depend on which tiles a
        # Gaussian's ellipse reaches: leave out tiles that a Gaussian near
        # that decision covers
        amb = (proj["visible"] == 1) & ((proj["margin_px"] < 1e-3) | (proj["margin_rel"] < 1e-5))
        tx_n, ty_n = oracle.tile_grid(cam, opts)
        unsure = np.zeros((ty_n, tx_n), bool)
        for x0, y0, x1, y1 in proj["rect"][amb]:
            unsure[y0:y1 + 1, x0:x1 + 1] = True
        tile_unsure = np.kron(unsure, np.ones((tile[1], tile[0]), bool))[:cam["height"], :cam["width"]]
        bad = (g["walked"].astype(np.int64) != ref["walked"]) & clear & ~tile_unsure
        assert not bad.any(), (ci, "walked", np.argwhere(bad)[:5])
        lens = (ranges[:, 1] - ranges[:, 0]).reshape(ty_n, tx_n)
        lens_px = np.kron(lens, np.ones((tile[1], tile[0]), np.int64))[:cam["height"], :cam["width"]]
        bad = (g["listed"].astype(np.int64) != lens_px) & ~tile_unsure
        assert not bad.any(), (ci, "listed", np.argwhere(bad)[:5])
        assert np.all(g["walked"] <= g["listed"])
        walked_checked += int((clear & ~tile_unsure).sum())
        assert g["m"].max() > 1
        # where many blend, most pixels need fewer than all of them
        many = ref["blended"] >= 20
        assert many.any() and (g["m"][many] < g["blended"][many]).mean() > 0.5
    assert walked_checked > 20000
    r.close()


def test_skew_rejects_bad_arguments(Renderer):
    from paper_2503_05168_gb300 import SeeleError
    sc, cams = _cases()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    for frac in (0.0, -0.5, 1.5):
        with pytest.raises(SeeleError):
            r.contribution_skew(frac)
    r.close()
