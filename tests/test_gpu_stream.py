"""Streamed scenes (Sec. 3.3 "Scene Prefetching", seele_load_scene_streamed):
only the shared Gaussians and a few view-cluster slots are resident; frames
load what their cameras select and prefetch the clusters of the linearly
extrapolated next pose.  Every frame must render the same Gaussians as the
whole scene resident with the cluster filter: equal visible and instance
counts, and equal images up to pixels where two Gaussians tie exactly in FP32
depth (record ids, which break such ties, differ between the layouts)."""
import math

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


def _path(n, width=160, height=90):
    """A smooth orbit at radius 4, a little above the scene."""
    return scenegen.orbit(n, 4.0, width, height, elevation_deg=8.0, phase=0.3)


def _frame(r, cams, **kw):
    r.set_cameras(cams)
    imgs, _ = parity.gpu_render(r, mode="cr", cluster_filter=True, opacity_filter=True, **kw)
    return imgs, r.last_stats["n_visible"], r.last_stats["n_instances"]


def _same(a, b, what):
    for x, y in zip(a, b):
        differ = np.any(x != y, axis=0)
        assert differ.mean() <= 2e-3, (what, differ.mean())


@pytest.mark.parametrize("graph,slots,chunk", [(False, 6, 0), (True, 6, 0), (False, 24, 1000), (True, 24, 1000)])
def test_streamed_frames_render_the_resident_scene(Renderer, graph, slots, chunk):
    """30% shared Gaussians, every other one in 3 neighbouring clusters (the
    precedence rule decides which slot draws it); one slot per cluster, or
    clusters cut into chunks of 1000."""
    sc, _ = scenegen.clusters_500k(n=20_000, width=160, height=90)
    path = _path(24)
    full = Renderer()
    full.load_scene(sc)
    st = Renderer()
    st.load_scene(sc, streamed_slots=slots, slot_gaussians=chunk, ahead=1)
    for i, cam in enumerate(path):
        a, va, ka = _frame(full, [cam])
        b, vb, kb = _frame(st, [cam], graph=graph)
        assert (va, ka) == (vb, kb), i
        _same(a, b, i)
    s = st.stream_stats()
    assert s["frames"] == len(path)
    m = sc["cluster_mask"] & np.uint32(0xFFFF)
    own = m[(m != 0) & (m != 0xFFFF)]
    sizes = np.array([np.count_nonzero(own & np.uint32(1 << k)) for k in range(16)])
    assert s["n_chunks"] == (16 if chunk == 0 else int((-(-sizes // chunk)).sum())), s
    # along a smooth path most selections were prefetched or stayed resident
    per = 1 if chunk == 0 else 4
    assert s["loads_sync"] <= per * (6 + len(path) // 4), s
    assert s["prefetch_hits"] > 0 and s["loads_prefetched"] > 0, s
    full.close()
    st.close()


def _balanced_clusters(means, C=16, shared_frac=0.02, seed=7):
    """Each Gaussian in one of C clusters of equal size by azimuth (2% shared);
    centroid c looks at the origin from radius 4 at its bin's middle azimuth."""
    rs = np.random.default_rng(seed)
    az = np.arctan2(means[:, 2].astype(np.float64), means[:, 0].astype(np.float64)) % (2 * math.pi)
    order = np.argsort(az, kind="stable")
    cl = np.empty(means.shape[0], np.int64)
    cl[order] = np.arange(means.shape[0]) * C // means.shape[0]
    mask = (np.uint32(1) << cl.astype(np.uint32)).astype(np.uint32)
    mask[rs.random(means.shape[0]) < shared_frac] = np.uint32(0xFFFFFFFF)
    mid = np.array([np.median(az[cl == c]) for c in range(C)])
    pos = np.stack([np.cos(mid), np.zeros(C), np.sin(mid)], 1)
    cen = np.concatenate([pos, -pos], 1) + rs.uniform(-1e-3, 1e-3, (C, 6))
    return mask, cen, 1.0


@pytest.mark.parametrize("slots,chunk", [(6, 0), (12, 620)])
def test_streamed_scene_holds_a_fraction_of_the_scene(Renderer, slots, chunk):
    """With few shared Gaussians and clusters of equal size, the resident part
    is the shared ones and 6 clusters' worth of slots (whole clusters, or
    half-cluster chunks)."""
    sc, _ = scenegen.clusters_500k(n=20_000, width=160, height=90)
    mask, cen, scale = _balanced_clusters(sc["means"])
    sc.update(cluster_mask=mask, centroids=cen, pos_scale=scale)
    path = _path(32)
    full = Renderer()
    full.load_scene(sc)
    st = Renderer()
    st.load_scene(sc, streamed_slots=slots, slot_gaussians=chunk, ahead=1)
    for i, cam in enumerate(path):
        a, va, ka = _frame(full, [cam])
        b, vb, kb = _frame(st, [cam])
        assert (va, ka) == (vb, kb), i
        _same(a, b, i)
    s = st.stream_stats()
    assert s["resident_bytes"] < 0.45 * s["full_bytes"], s
    # the selection changes 11 times along the path; after the first frame's
    # four clusters, nearly every new one was prefetched in time
    per = 1 if chunk == 0 else 2
    assert s["loads_sync"] <= per * (4 + 3), s
    assert s["prefetch_hits"] >= per * 8, s
    full.close()
    st.close()


def test_streamed_two_camera_frames(Renderer):
    sc, _ = scenegen.clusters_500k(n=20_000, width=160, height=90)
    a_path, b_path = _path(10), scenegen.orbit(10, 4.0, 120, 80, elevation_deg=-5.0, phase=2.0)
    full = Renderer()
    full.load_scene(sc)
    st = Renderer()
    st.load_scene(sc, streamed_slots=10, ahead=2)
    for i in range(10):
        cams = [a_path[i], b_path[i]]
        a, va, ka = _frame(full, cams)
        b, vb, kb = _frame(st, cams)
        assert (va, ka) == (vb, kb), i
        _same(a, b, i)
    full.close()
    st.close()


def test_streamed_scene_rules(Renderer):
    from paper_2503_05168_gb300 import SeeleError
    sc, cams = scenegen.clusters_500k(n=5_000, width=64, height=48)
    r = Renderer()
    r.load_scene(sc, streamed_slots=4)
    r.set_cameras(cams[:1])
    with pytest.raises(SeeleError):  # the cluster filter is required
        r.render(mode="cr")
    r.render(mode="cr", cluster_filter=True)
    import torch
    with pytest.raises(SeeleError):  # gradients need the whole scene
        r.render_backward(torch.zeros(3 * 64 * 48, device=r.device))
    r.set_cameras(cams[:2])  # two cameras far apart select more clusters than 4 slots
    with pytest.raises(SeeleError):
        r.render(mode="cr", cluster_filter=True, n_neighbors=3)
    with pytest.raises(SeeleError):
        r.load_scene({k: v for k, v in sc.items() if k != "cluster_mask"}, streamed_slots=4)
    r.load_scene(sc)  # back to a resident scene
    r.set_cameras(cams[:1])
    r.render(mode="cr", cluster_filter=True)
    with pytest.raises(SeeleError):
        r.stream_stats()
    r.close()
