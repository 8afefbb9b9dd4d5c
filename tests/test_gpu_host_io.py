"""Scene loads from every kind of memory and renders into host memory: the
repack (caller layout -> planes) at every SH degree and a ragged Gaussian
count against the oracle, pageable / page-locked / device sources giving
the same scene, and asynchronous and graph renders into page-locked host
images."""
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


def _scene(deg, n=3001, seed=4):
    # 3001 = 23 repack blocks of 128 and a tail of 57
    sc, cams = scenegen.uniform_10k(seed=seed, n=n)
    nc = (deg + 1) ** 2
    sc["sh"] = np.ascontiguousarray(sc["sh"][:, :nc, :])
    sc["sh_degree"] = deg
    return sc, cams


def _source(sc, kind):
    import torch
    if kind == "numpy":
        return sc
    if kind == "borrow":   # device arrays read in place
        return _source(sc, "device")
    out = {}
    for k, v in sc.items():
        if k in ("means", "log_scales", "quats", "opacity_logits", "sh", "cluster_mask"):
            t = torch.from_numpy(np.ascontiguousarray(v))
            out[k] = t.pin_memory() if kind == "pinned" else t.cuda()
        else:
            out[k] = v
    return out


@pytest.mark.parametrize("kind", ["numpy", "pinned", "device", "borrow"])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_records_match_oracle_at_every_sh_degree(Renderer, deg, kind):
    sc, cams = _scene(deg)
    r = Renderer()
    r.load_scene(_source(sc, kind), borrow=(kind == "borrow"))
    r.set_cameras(cams)
    parity.gpu_render(r)
    d = parity.debug_numpy(r)
    proj = oracle.preprocess(oracle.Scene64.from_scene(sc), cams[0], oracle.Options())
    vis_g = d["tiles_touched"] > 0
    vis_o = proj["visible"] == 1
    clear = (proj["margin_px"] >= 1e-3) & (proj["margin_rel"] >= 1e-5)
    assert np.array_equal(vis_g[clear], vis_o[clear])
    both = vis_g & vis_o & clear
    assert both.sum() > 2500
    u, v, con, o, rgb = parity.records_to_proj(d["records"][both])
    np.testing.assert_allclose(u, proj["uv"][both, 0], atol=2e-3)
    np.testing.assert_allclose(v, proj["uv"][both, 1], atol=2e-3)
    cn = np.linalg.norm(proj["conic"][both], axis=1, keepdims=True)
    assert np.max(np.abs(con - proj["conic"][both]) / cn) < 1e-3
    np.testing.assert_allclose(o, proj["opacity"][both], rtol=1e-5)
    np.testing.assert_allclose(rgb, proj["rgb"][both], atol=1e-5)
    r.close()


@pytest.mark.parametrize("spatial", [False, True])
def test_load_sources_give_the_same_scene(Renderer, spatial):
    sc, cams = scenegen.clusters_500k(n=20_001, width=200, height=120, n_cams=2)
    imgs, recs = [], []
    for kind in ("numpy", "pinned", "device"):
        r = Renderer()
        r.load_scene(_source(sc, kind), spatial=spatial)
        r.set_cameras(cams)
        im, _ = parity.gpu_render(r, mode="cr", cluster_filter=True)
        imgs.append(im)
        recs.append(parity.debug_numpy(r)["records"])
        r.close()
    for k in (1, 2):
        assert np.array_equal(recs[0].view(np.uint32), recs[k].view(np.uint32))
        for x, y in zip(imgs[0], imgs[k]):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_async_and_graph_renders_into_page_locked_host(Renderer):
    import torch
    from paper_2503_05168_gb300 import SeeleError
    sc, cams = scenegen.clusters_500k(n=20_000, width=160, height=90, n_cams=3)
    r = Renderer()
    r.load_scene(sc, spatial=True)
    npix = 160 * 90
    refs = []
    for c in cams:
        r.set_cameras([c])
        T = torch.empty(npix, device="cuda")
        img = r.render(mode="cr", opacity_filter=True, out_T=T)
        torch.cuda.synchronize()
        refs.append((img.cpu(), T.cpu()))
    host = torch.full((3 * npix,), float("nan")).pin_memory()
    host_T = torch.full((npix,), float("nan")).pin_memory()
    for flags in (dict(sync=True), dict(sync=False), dict(sync=False, graph=True)):
        opts = r.make_options(mode="cr", opacity_filter=True, **flags)
        for rep in range(2):
            for c, (ref, ref_T) in zip(cams, refs):
                r.set_cameras([c])
                r.render(out=host, out_T=host_T, options=opts)
                r.synchronize()
                assert torch.equal(host.view(torch.int32), ref.view(torch.int32)), (flags, rep)
                assert torch.equal(host_T.view(torch.int32), ref_T.view(torch.int32)), (flags, rep)
                host.fill_(float("nan"))
                host_T.fill_(float("nan"))
    # pageable host memory cannot be written asynchronously
    pageable = np.empty(3 * npix, dtype=np.float32)
    with pytest.raises(SeeleError):
        r.render(out=pageable, mode="cr", sync=False)
    with pytest.raises(SeeleError):
        r.render(out=pageable, mode="cr", sync=False, graph=True)
    r.render(out=pageable, mode="cr", opacity_filter=True)   # synchronous: fine
    assert np.array_equal(pageable.view(np.uint32), refs[-1][0].numpy().view(np.uint32))
    r.close()


@pytest.mark.parametrize("deg", [1, 3])
def test_borrowed_arrays_in_place_or_repacked(Renderer, deg):
    """A BORROW scene is read in place when its quaternion and SH arrays are
    16-byte aligned and repacked first when they are not: the same bits as
    the copied scene either way, forward and backward."""
    import torch
    sc, cams = _scene(deg, n=5001)
    ref = Renderer()
    ref.load_scene(sc)
    ref.set_cameras(cams)
    img_ref, _ = parity.gpu_render(ref, mode="cr")
    w = torch.from_numpy(np.random.default_rng(5).standard_normal(3 * 256 * 256).astype(np.float32)).cuda()
    g_ref = {k: v.cpu().numpy() for k, v in ref.render_backward(w).items()}
    dev = _source(sc, "device")
    # the same arrays one float into a larger buffer: 4-byte aligned only
    shifted = dict(dev)
    for k in ("quats", "sh"):
        buf = torch.zeros(dev[k].numel() + 1, device="cuda")
        buf[1:] = dev[k].reshape(-1)
        shifted[k] = buf[1:].view(dev[k].shape)
        assert shifted[k].data_ptr() % 16 == 4
    for arrays in (dev, shifted):
        r = Renderer()
        r.load_scene(arrays, borrow=True)
        r.set_cameras(cams)
        img, _ = parity.gpu_render(r, mode="cr")
        for x, y in zip(img, img_ref):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
        g = {k: v.cpu().numpy() for k, v in r.render_backward(w).items()}
        for k in g_ref:
            # float atomics add the per-pixel terms in any order
            assert np.max(np.abs(g[k] - g_ref[k])) <= 1e-5 * (np.abs(g_ref[k]).max() + 1e-30), k
        r.close()
    ref.close()
