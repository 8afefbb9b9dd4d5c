"""Contexts sharing one resident scene (seele_share_scene): the same frames
as the context that loaded it, frames of both in flight at once on their own
streams, and a scene that outlives the context that loaded it."""
import numpy as np
import pytest

import scenegen
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _same_bits(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("spatial", [False, True])
@pytest.mark.parametrize("kw", [dict(mode="plain"), dict(mode="cr", opacity_filter=True),
                                dict(mode="cr", cluster_filter=True, binning="tiles")])
def test_shared_scene_renders_the_same_bits(Renderer, spatial, kw):
    sc, cams = scenegen.clusters_500k(n=30_000, width=200, height=120, n_cams=3)
    a, b = Renderer(), Renderer()
    a.load_scene(sc, spatial=spatial)
    b.share_scene(a)
    for r in (a, b):
        r.set_cameras(cams)
    ia, Ta = parity.gpu_render(a, **kw)
    ib, Tb = parity.gpu_render(b, **kw)
    _same_bits(ia, ib)
    _same_bits(Ta, Tb)
    assert a.last_stats["n_instances"] == b.last_stats["n_instances"]
    if spatial:
        da, db = parity.debug_numpy(a), parity.debug_numpy(b)
        assert np.array_equal(da["scene_order"], db["scene_order"])
    a.close()
    b.close()


def test_frames_in_flight_on_two_streams(Renderer):
    """Two renderers on their own streams take alternate frames, captured
    graphs replayed without host synchronisation; every frame equals the
    one a single renderer draws."""
    import torch
    sc, cams = scenegen.clusters_500k(n=40_000, width=320, height=180, n_cams=8)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    rs = [Renderer(stream=s) for s in streams]
    rs[0].load_scene(sc, spatial=True)
    rs[1].share_scene(rs[0])
    n_frames = 16
    npix = 3 * 320 * 180
    outs = [torch.full((npix,), float("nan"), device="cuda") for _ in range(n_frames)]
    opts = [r.make_options(mode="cr", opacity_filter=True, sync=False, graph=True) for r in rs]
    torch.cuda.synchronize()
    for i in range(n_frames):
        r = rs[i % 2]
        r.set_cameras([cams[i % 8]])
        r.render(out=outs[i], options=opts[i % 2])
    for r in rs:
        r.synchronize()
    torch.cuda.synchronize()
    ref = Renderer()
    ref.share_scene(rs[0])
    for i in range(n_frames):
        ref.set_cameras([cams[i % 8]])
        img = ref.render(mode="cr", opacity_filter=True)
        torch.cuda.synchronize()
        assert torch.equal(img.view(torch.int32), outs[i].view(torch.int32)), i
    for r in rs + [ref]:
        r.close()


def test_shared_scene_outlives_its_loader(Renderer):
    """Reloading or destroying the context that loaded the scene leaves the
    sharing context's scene as it was shared."""
    sx, cams = scenegen.clusters_500k(n=20_000, width=160, height=90, n_cams=2)
    sy, _ = scenegen.clusters_500k(n=12_000, width=160, height=90, n_cams=2, seed=5)
    a, b = Renderer(), Renderer()
    a.load_scene(sx, spatial=True)
    a.set_cameras(cams)
    ref, _ = parity.gpu_render(a, mode="cr")
    b.share_scene(a)
    b.set_cameras(cams)
    a.load_scene(sy)            # a lets go of the first scene
    iy, _ = parity.gpu_render(a, mode="cr")
    ib, _ = parity.gpu_render(b, mode="cr")
    _same_bits(ref, ib)
    assert any(np.any(x != y) for x, y in zip(iy, ib))
    a.close()                   # b alone holds the first scene
    c = Renderer()
    c.share_scene(b)            # shared again from a context that shares it
    c.set_cameras(cams)
    ic, _ = parity.gpu_render(c, mode="cr")
    ib, _ = parity.gpu_render(b, mode="cr")
    _same_bits(ref, ic)
    _same_bits(ref, ib)
    b.load_scene(sy)            # and c keeps it after b moves on
    ic, _ = parity.gpu_render(c, mode="cr")
    _same_bits(ref, ic)
    b.close()
    c.close()


def test_shared_borrowed_scene(Renderer):
    import torch
    sc, cams = scenegen.uniform_10k()
    dev = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v)
           for k, v in sc.items()}
    a, b = Renderer(), Renderer()
    a.load_scene(dev, borrow=True)
    b.share_scene(a)
    for r in (a, b):
        r.set_cameras(cams)
    ia, _ = parity.gpu_render(a, mode="cr")
    ib, _ = parity.gpu_render(b, mode="cr")
    _same_bits(ia, ib)
    # the caller's arrays are read every frame: a change shows in both
    dev["opacity_logits"].fill_(-30.0)
    ia, _ = parity.gpu_render(a, mode="cr")
    ib, _ = parity.gpu_render(b, mode="cr")
    for x, y in zip(ia, ib):
        assert x.max() == 0.0 and y.max() == 0.0
    a.close()
    b.close()


def test_shared_scene_gradients_and_builder(Renderer):
    import torch
    sc, cams = scenegen.uniform_10k()
    a, b = Renderer(), Renderer()
    a.load_scene(sc, spatial=True)
    b.share_scene(a)
    for r in (a, b):
        r.set_cameras(cams)
        r.render(mode="cr")
    w = torch.from_numpy(np.random.default_rng(3).standard_normal(3 * 256 * 256).astype(np.float32)).cuda()
    ga, gb = a.render_backward(w), b.render_backward(w)
    for k in ga:
        x, y = ga[k].cpu().numpy(), gb[k].cpu().numpy()
        # float atomics add the per-pixel terms in any order
        assert np.max(np.abs(x - y)) <= 1e-4 * (np.abs(x).max() + 1e-30), k
    poses = scenegen.orbit(8, 3.0, 64, 64)
    ma = a.build_view_clusters(poses, n_clusters=4, top_k=8)
    mb = b.build_view_clusters(poses, n_clusters=4, top_k=8)
    assert np.array_equal(ma["mask"], mb["mask"])
    a.close()
    b.close()


def test_share_scene_rules(Renderer):
    from paper_2503_05168_gb300 import SeeleError
    sc, cams = scenegen.clusters_500k(n=5_000, width=64, height=48)
    a, b = Renderer(), Renderer()
    with pytest.raises(SeeleError):   # nothing loaded yet
        b.share_scene(a)
    with pytest.raises(SeeleError):   # itself
        a.share_scene(a)
    a.load_scene(sc, streamed_slots=4)
    with pytest.raises(SeeleError):   # a streamed scene's slots change every frame
        b.share_scene(a)
    a.load_scene(sc)
    b.share_scene(a)
    b.set_cameras(cams[:1])
    b.render(mode="cr", cluster_filter=True)
    a.close()
    b.close()
