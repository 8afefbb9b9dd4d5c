"""GPU backward (raster + preprocessing kernels, through the C ABI) against the
FP64 oracle's analytic gradients, which tests/test_oracle_grad.py pins to
central finite differences.

Bar (relative error 1e-3, as the plan states for gradients): for every
parameter group (means, log-scales, quaternions, opacity logits, SH) the
relative L2 error is <= 1e-3, and every element is within
1e-3 * (|g| + rms of its group) except a few elements whose Gaussians cover a
pixel where an FP32 decision (support, alpha_theta, leader, stop) flips
against FP64 -- at most 0.1% of a group (measured: ~3e-5, and ~1e-5
relative L2).
"""
import numpy as np
import pytest

import oracle
import scenegen
from tests import parity

pytestmark = pytest.mark.gpu

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _compare(gpu, ref):
    rep = {}
    ok = True
    for k in GROUPS:
        a = gpu[k].reshape(-1).astype(np.float64)
        b = ref[k].reshape(-1)
        rms = np.sqrt(np.mean(b ** 2))
        l2 = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        bad = np.abs(a - b) > 1e-3 * (np.abs(b) + rms)
        rep[k] = dict(rel_l2=float(l2), bad_frac=float(bad.mean()), n=int(b.size))
        ok &= (l2 <= 1e-3) and (bad.mean() <= 1e-3)
    return ok, rep


@pytest.mark.parametrize("mode,group,tile", [("plain", (2, 2), (16, 16)), ("cr", (2, 2), (16, 16)),
                                             ("cr", (4, 4), (16, 16)), ("cr", (2, 2), (8, 8))])
def test_backward_matches_oracle_analytic(Renderer, mode, group, tile):
    import torch
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    r.render(mode=mode, group=group, tile=tile)
    rs = np.random.default_rng(7)
    w = rs.standard_normal((3, 256, 256))
    g = r.render_backward(torch.from_numpy(w.reshape(-1).astype(np.float32)).cuda())
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in g.items()}
    ref = oracle.backward(oracle.Scene64.from_scene(sc), cams[0],
                          oracle.Options(cr=(mode == "cr"), group_w=group[0], group_h=group[1], tile_w=tile[0],
                                         tile_h=tile[1]), w)
    ok, rep = _compare(gpu, ref)
    print(mode, rep)
    assert ok, rep
    r.close()


def test_autograd_function_equals_direct_backward(Renderer):
    import torch
    from paper_2503_05168_gb300 import render
    sc, cams = scenegen.uniform_10k(n=3000, width=96, height=80)
    cams[0]["fx"] = cams[0]["fy"] = 90.0
    r = Renderer()
    r.set_cameras(cams)
    params = {k: torch.from_numpy(np.ascontiguousarray(sc[k])).cuda().requires_grad_(True)
              for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    img = render(r, **params, sh_degree=3, mode="cr")
    w = torch.randn_like(img)
    (img * w).sum().backward()
    r2 = Renderer()
    r2.load_scene(sc)
    r2.set_cameras(cams)
    img2 = r2.render(mode="cr")
    torch.testing.assert_close(img.detach(), img2, rtol=0, atol=0)
    g2 = r2.render_backward(w)
    # float atomics sum the per-pixel terms in a nondeterministic order
    for k, p in params.items():
        torch.testing.assert_close(p.grad, g2[k].reshape(p.shape), rtol=1e-5, atol=1e-6)
    r.close()
    r2.close()


def test_backward_of_camera_batch_is_sum_over_cameras(Renderer):
    import torch
    sc, _ = scenegen.uniform_10k(n=4000)
    cams = [scenegen.look_at((0.4 * i, -0.2, -3), (0, 0, 0), w, h) for i, (w, h) in enumerate([(64, 48), (100, 70)])]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    img = r.render(mode="cr")
    w = torch.randn_like(img)
    gb = r.render_backward(w)
    acc = None
    off = 0
    for c in cams:
        k = 3 * c["width"] * c["height"]
        r.set_cameras([c])
        r.render(mode="cr")
        gs = r.render_backward(w[off:off + k].contiguous())
        acc = gs if acc is None else {n: acc[n] + gs[n] for n in acc}
        off += k
    for n in GROUPS:
        torch.testing.assert_close(gb[n], acc[n], rtol=1e-4, atol=1e-6)
    r.close()


@pytest.mark.parametrize("mode", ["plain", "cr"])
def test_backward_of_long_lists_walked_in_chunks(Renderer, mode):
    """Tile lists of thousands of entries that pixels walk deep into (faint,
    wide, dense Gaussians): the backward pass walks them in 256-entry chunks,
    each CTA starting from the forward pass's transmittance checkpoint.
    Gradients match the oracle, walked in chunks and walked whole (a
    counting render writes no checkpoints)."""
    import torch
    sc, cams = scenegen.uniform_10k(seed=3, n=20_000, width=96, height=96)
    sc["opacity_logits"] = sc["opacity_logits"] - np.float32(3.0)
    sc["log_scales"] = sc["log_scales"] + np.float32(1.0)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    w = np.random.default_rng(9).standard_normal((3, 96, 96))
    wt = torch.from_numpy(w.reshape(-1).astype(np.float32)).cuda()
    ref = oracle.backward(oracle.Scene64.from_scene(sc), cams[0], oracle.Options(cr=(mode == "cr")), w)
    grads = {}
    for walk, count in (("chunks", False), ("whole", True)):
        r.render(mode=mode, binning="tiles", count=count)
        d = parity.debug_numpy(r)
        nc = d["n_contrib"].reshape(96, 96)
        assert nc.max() > 3 * 256   # pixels walk past several checkpoints
        g = r.render_backward(wt)
        torch.cuda.synchronize()
        grads[walk] = {k: v.cpu().numpy() for k, v in g.items()}
        ok, rep = _compare(grads[walk], ref)
        assert ok, (walk, rep)
    r.close()
