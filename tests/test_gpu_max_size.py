"""The largest scene the boundary accepts: n = 65535 * 256 = 16,776,960
Gaussians (record ids fill 24 bits, the limit of the count packed beside
them in the depth sort), one 256x256 camera, the benchmark's launch
configuration (CR + opacity-aware filtering, block binning).  Checked
bit-identical to the same frame binned by tiles, per-Gaussian visibility and
tile counts against the oracle for every Gaussian, and binning and blending
against the oracle on sampled tiles; one Gaussian more is refused."""
import numpy as np
import pytest

import oracle
import scenegen
from tests import parity

pytestmark = pytest.mark.gpu

N_MAX = 65535 * 256


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _scene(n, seed=11):
    # the attribute distributions of the 10k config at SH degree 0 (host
    # memory stays under 1 GB), sub-pixel to few-pixel footprints
    r = np.random.default_rng(seed)
    q = r.standard_normal((n, 4), dtype=np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return dict(means=r.uniform(-1, 1, (n, 3)).astype(np.float32),
                log_scales=(np.float32(np.log(0.004)) + np.float32(0.5) * r.standard_normal((n, 3), dtype=np.float32)),
                quats=q, opacity_logits=np.float32(1.5) * r.standard_normal(n, dtype=np.float32),
                sh=(np.float32(0.5) + np.float32(0.2) * r.standard_normal((n, 1, 3), dtype=np.float32)),
                sh_degree=0)


def test_maximum_gaussian_count(Renderer):
    from paper_2503_05168_gb300 import SeeleError
    sc = _scene(N_MAX)
    cam = scenegen.look_at((0.3, -0.2, -3.0), (0, 0, 0), 256, 256)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras([cam])
    img = r.images(r.render(mode="cr", opacity_filter=True))[0].cpu().numpy()
    img_t = r.images(r.render(mode="cr", opacity_filter=True, binning="tiles"))[0].cpu().numpy()
    np.testing.assert_array_equal(img, img_t)
    d = parity.debug_numpy(r)

    s64 = oracle.Scene64.from_scene(sc)
    opts = parity.oracle_options("cr", opacity_filter=True)
    proj = oracle.preprocess(s64, cam, opts, nthreads=16)
    clear = (proj["margin_px"] >= 1e-3) & (proj["margin_rel"] >= 1e-5)
    assert clear.mean() > 0.99
    vis_o = proj["visible"] == 1
    touched = d["tiles_touched"].astype(np.int64)
    assert touched.shape[0] == N_MAX
    assert np.array_equal((touched > 0)[clear], vis_o[clear])
    both = clear & vis_o
    assert both.sum() > N_MAX // 2
    assert np.array_equal(touched[both], proj["ntiles"][both])
    # the last Gaussians (ids near 2^24) are among the binned ones
    assert vis_o[-1000:].any() and (touched[-1000:] > 0).any()

    tx_n, ty_n = oracle.tile_grid(cam, opts)
    rng = d["tile_ranges"].astype(np.int64)
    rs = np.random.default_rng(7)
    tiles = np.concatenate([rs.choice(tx_n * ty_n, 6, replace=False), [0, tx_n * ty_n - 1],
                            [int(np.argmax(rng[:, 1] - rng[:, 0]))]])
    ref, lists, (sub, gid, ranges) = parity.oracle_render_tiles(proj, cam, opts, tiles)
    W = cam["width"]
    pix = []
    for t in np.unique(tiles):
        tx, ty = t % tx_n, t // tx_n
        yy, xx = np.mgrid[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16]
        pix.append((yy * W + xx).reshape(-1))
    rep = parity.check_render(img, None, ref, sub, gid, ranges, cam, opts, pixels=np.concatenate(pix))
    assert rep["ok"], str(rep)
    for t in np.unique(tiles):
        g_gpu = d["inst_record"][rng[t, 0]:rng[t, 1]].astype(np.int64)
        g_or = lists[int(t)]
        assert set(g_gpu[clear[g_gpu]].tolist()) == set(g_or[clear[g_or]].tolist()), int(t)
    del d, proj, s64

    # one Gaussian more than the boundary accepts
    big = {k: (np.concatenate([v, v[:1]]) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    with pytest.raises(SeeleError, match="ERR_ARG"):
        r.load_scene(big)
    r.close()
