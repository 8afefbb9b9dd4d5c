"""seele_sort_tile_instances_noalloc: the tile-instance sort for callers that
cannot allocate device memory.

A host that owns the whole device memory budget, or a real-time loop in which
an allocation (which can synchronise the device) would stall a frame, cannot
let a library call cudaMalloc.  This entry point keeps its scratch in a fixed
array inside the library instead.  The test feeds it the tile instances of a
real render in front-to-back order -- what the render path emits -- and
checks the per-tile lists and ranges against the ones seele_render built (read
through seele_get_debug_view), on two calls in a row, for a frame with fewer
than 256 tiles (one radix pass) and one with more (two passes).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _front_to_back_instances(d, tiles_x):
    """Instances in the order the render path emits them: visible records by
    (fp32 depth, record id), each record's tiles in row-major order.  The
    (tile, record) pairs are the render's own sorted lists, reordered."""
    rec = d["inst_record"].astype(np.int64)
    tile = d["inst_tile"].astype(np.int64)
    dbits = d["depth"].view(np.uint32).astype(np.int64)
    order = np.lexsort((tile, rec, dbits[rec]))
    return tile[order].astype(np.uint32), rec[order].astype(np.uint32)


def _call(lib, stream, tiles, recs, n_tiles):
    import torch
    dev = torch.device("cuda")
    t = torch.from_numpy(tiles.view(np.int32)).to(dev)
    r = torch.from_numpy(recs.view(np.int32)).to(dev)
    out = torch.full((tiles.size,), -7, dtype=torch.int32, device=dev)
    start = torch.zeros(n_tiles, dtype=torch.int32, device=dev)
    end = torch.zeros(n_tiles, dtype=torch.int32, device=dev)
    st = lib.seele_sort_tile_instances_noalloc(
        ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(r.data_ptr()), tiles.size, n_tiles,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(start.data_ptr()), ctypes.c_void_p(end.data_ptr()),
        ctypes.c_void_p(stream))
    return st, out.cpu().numpy().view(np.uint32), start.cpu().numpy().view(np.uint32), end.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("width,height", [(256, 256), (640, 480)])
def test_noalloc_sort_matches_the_render_path_twice(Renderer, width, height):
    import torch
    from paper_2503_05168_gb300 import lib
    sc, cams = scenegen.uniform_10k(width=width, height=height)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    r.render(mode="cr", opacity_filter=True, binning="tiles")
    torch.cuda.synchronize()
    d = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.debug_view().items()}
    tiles_x = (width + 15) // 16
    n_tiles = tiles_x * ((height + 15) // 16)
    assert n_tiles == d["n_tiles"]
    tiles, recs = _front_to_back_instances(d, tiles_x)
    assert tiles.size == d["n_instances"] > 0
    exp_rec = d["inst_record"].view(np.uint32)
    exp_rng = d["tile_ranges"].astype(np.int64)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        st, got, start, end = _call(lib(), stream, tiles, recs, n_tiles)
        assert st == 0
        np.testing.assert_array_equal(got, exp_rec)
        nonempty = exp_rng[:, 1] > exp_rng[:, 0]
        np.testing.assert_array_equal(start[nonempty], exp_rng[nonempty, 0])
        np.testing.assert_array_equal(end[nonempty], exp_rng[nonempty, 1])
        assert np.all(start[~nonempty].astype(np.int64) >= end[~nonempty])
    r.close()


def _stable_reference(tiles, recs, n_tiles):
    order = np.argsort(tiles, kind="stable")
    counts = np.bincount(tiles, minlength=n_tiles)
    start = np.concatenate([[0], np.cumsum(counts)[:-1]])
    return recs[order], start, start + counts, counts > 0


@pytest.mark.parametrize("n,n_tiles", [(1 << 20, 1 << 16), (300_007, 8160), (0, 17), (5000, 200)])
def test_noalloc_sort_matches_a_stable_argsort_twice(Renderer, n, n_tiles):
    """Random tile ids at the limits (2^20 instances over 2^16 tiles: 16 scan
    blocks, two radix passes), a mid size, a single pass and no instances at
    all, each sorted twice in a row so that look-back entries left by the
    previous call are met too."""
    import torch
    from paper_2503_05168_gb300 import lib
    rs = np.random.default_rng(n + n_tiles)
    tiles = rs.integers(0, n_tiles, n).astype(np.uint32)
    recs = rs.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    exp_rec, exp_start, exp_end, nonempty = _stable_reference(tiles, recs, n_tiles)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        st, got, start, end = _call(lib(), stream, tiles, recs, n_tiles)
        assert st == 0
        np.testing.assert_array_equal(got, exp_rec)
        np.testing.assert_array_equal(start[nonempty], exp_start[nonempty])
        np.testing.assert_array_equal(end[nonempty], exp_end[nonempty])
        assert np.all(start[~nonempty].astype(np.int64) >= end[~nonempty])


def test_noalloc_sort_refuses_bad_tile_ids_and_misaligned_input(Renderer):
    """A tile id >= n_tiles is found on the device: nothing is sorted, every
    list stays empty and the call returns SEELE_ERR_ARG; a tile-id pointer
    that is not 16-byte aligned is refused before any GPU work."""
    import torch
    from paper_2503_05168_gb300 import lib
    stream = torch.cuda.current_stream().cuda_stream
    tiles = np.arange(1000, dtype=np.uint32) % 64
    tiles[617] = 64
    recs = np.arange(1000, dtype=np.uint32)
    st, got, start, end = _call(lib(), stream, tiles, recs, 64)
    assert st == 1
    assert np.all(start.astype(np.int64) >= end) and np.all(got == np.uint32(0xFFFFFFF9))
    t = torch.from_numpy((tiles % 64).view(np.int32)).cuda()
    r = torch.from_numpy(recs.view(np.int32)).cuda()
    out = torch.zeros(1000, dtype=torch.int32, device="cuda")
    se = torch.zeros(64, dtype=torch.int32, device="cuda")
    st = lib().seele_sort_tile_instances_noalloc(
        ctypes.c_void_p(t[1:].data_ptr()), ctypes.c_void_p(r.data_ptr()), 999, 64, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(se.data_ptr()), ctypes.c_void_p(se.data_ptr()), ctypes.c_void_p(stream))
    assert st == 1
    # and the next ordinary call works
    st, got, start, end = _call(lib(), stream, tiles % 64, recs, 64)
    assert st == 0
    np.testing.assert_array_equal(got, _stable_reference(tiles % 64, recs, 64)[0])


def test_noalloc_sort_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2503_05168_gb300 import _abi, lib
    torch.cuda.init()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    L = lib()
    assert L.seele_sort_tile_instances_noalloc(p, p, _abi.NOALLOC_MAX_INSTANCES + 1, 16, p, p, p, None) == 1
    assert L.seele_sort_tile_instances_noalloc(p, p, 4, _abi.NOALLOC_MAX_TILES + 1, p, p, p, None) == 1
    assert L.seele_sort_tile_instances_noalloc(p, p, 4, 0, p, p, p, None) == 1
