"""The checked build (SEELE_CHECKED, libseele_checked.so) renders the same frames.

The checked build validates every index the rasterizer gathers with (list
ranges against the instance count, record ids against the frame's records,
block ids against the frame's blocks) before using it, and reports a bad one
as SEELE_ERR_INTERNAL instead of reading out of bounds -- the stand-in for a
memory checker on this pool.  The same script runs in two processes, one on
each build (selected with SEELE_LIBRARY), and the images and transmittances
must be identical bit for bit, with no check firing.  Gradients are summed
over pixels with float atomics, whose order differs from run to run, so they
are compared within a relative L2 of 1e-6 instead.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[2])
import scenegen
from paper_2503_05168_gb300 import Renderer, _abi
out = {"lib": np.array(_abi.LIB_PATH)}
sc, cams = scenegen.uniform_10k()
extra = scenegen.look_at((0.6, -0.3, -3.2), (0, 0, 0), 100, 70)
r = Renderer()
r.load_scene(sc)
r.set_cameras([cams[0], extra])
for name, kw in (("cr_blocks", dict(mode="cr", opacity_filter=True)),
                 ("plain_tiles", dict(mode="plain", binning="tiles")),
                 ("cr_queue", dict(mode="cr", schedule="queue", batch_depth=1)),
                 ("cr_8x8", dict(mode="cr", tile=(8, 8), binning="tiles"))):
    T = torch.empty(r.n_pixels, device="cuda")
    img = r.render(out_T=T, **kw)
    out[name] = img.cpu().numpy()
    out[name + "_T"] = T.cpu().numpy()
r.set_cameras([cams[0]])
img = r.render(mode="cr", binning="tiles")
g = r.render_backward(torch.ones_like(img) / img.numel())
for k, v in g.items():
    out["grad_" + k] = v.cpu().numpy()
np.savez(sys.argv[1], **out)
print("ok")
'''


def _run(tmp_path, lib, tag):
    script = tmp_path / "frames.py"
    script.write_text(SCRIPT)
    dest = tmp_path / f"{tag}.npz"
    env = dict(os.environ, SEELE_LIBRARY=lib)
    res = subprocess.run([sys.executable, str(script), str(dest), ROOT], env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0 and "ok" in res.stdout, res.stderr[-3000:]
    return np.load(dest)


def test_checked_build_renders_the_same_frames(tmp_path):
    from paper_2503_05168_gb300.builder import build
    plain_lib = build()
    checked_lib = build(checked=True)
    a = _run(tmp_path, plain_lib, "plain")
    b = _run(tmp_path, checked_lib, "checked")
    assert str(b["lib"]).endswith("libseele_checked.so") and str(a["lib"]).endswith("libseele.so")
    keys = [k for k in a.files if k != "lib"]
    assert len(keys) >= 12
    for k in keys:
        if k.startswith("grad_"):
            x, y = a[k].astype(np.float64), b[k].astype(np.float64)
            assert np.linalg.norm(x - y) <= 1e-6 * np.linalg.norm(x), k
            assert np.abs(x).max() > 0, k
        else:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
