"""Pin of the oracle's analytic backward against FP64 central finite differences.

The loss is L = sum(w * rgb) with fixed random weights w, so dL/drgb = w.  A
parameter is re-drawn when a discrete decision (visibility, support, alpha
threshold, stop, clamps, CR leader skips) differs between theta - h, theta and
theta + h: the gradient holds those decisions fixed (Sec. 3.5).
"""
import numpy as np
import pytest

import oracle
import scenegen

FIELDS = [("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)]


def _forward(s64, cam, opts, w):
    r, proj, _, gid, ranges = oracle.render(s64, cam, opts, nthreads=8)
    loss = float((w * r.rgb).sum())
    c = r.counters
    sig = (r.ncontrib.tobytes(), c["blended"], c["terminated"], c["clamped"], c["leader_skips"],
           proj["visible"].tobytes(), np.signbit(proj["rgb_raw"]).tobytes(), c["alpha_evals"])
    return loss, sig, proj, gid, ranges


def _fd_check(opts, nparams, seed, n=10_000, W=256, H=256):
    sc, cams = scenegen.uniform_10k(n=n, width=W, height=H)
    cam = cams[0]
    s64 = oracle.Scene64.from_scene(sc)
    rs = np.random.default_rng(seed)
    w = rs.standard_normal((3, H, W))
    L0, sig0, proj, gid, ranges = _forward(s64, cam, opts, w)
    g = oracle.backward(s64, cam, opts, w, proj=proj, gid=gid, ranges=ranges)
    vis = np.nonzero(proj["visible"])[0]
    checked, errs = 0, []
    tries = 0
    while checked < nparams:
        tries += 1
        assert tries < 8 * nparams, "too many re-draws"
        gi = int(rs.choice(vis))
        name, size = FIELDS[rs.integers(len(FIELDS))]
        k = int(rs.integers(size))
        arr = getattr(s64, name)
        flat = arr.reshape(n, -1)
        theta = flat[gi, k]
        h = 1e-6 * max(1.0, abs(theta))
        flat[gi, k] = theta + h
        Lp, sigp, *_ = _forward(s64, cam, opts, w)
        flat[gi, k] = theta - h
        Lm, sigm, *_ = _forward(s64, cam, opts, w)
        flat[gi, k] = theta
        if sigp != sig0 or sigm != sig0:
            continue
        fd = (Lp - Lm) / (2 * h)
        an = g[name].reshape(n, -1)[gi, k]
        errs.append((name, fd, an))
        checked += 1
    return errs


@pytest.mark.parametrize("opts,nparams,seed", [(oracle.Options(), 64, 0), (oracle.Options(cr=True), 24, 1)])
def test_analytic_backward_matches_central_differences(opts, nparams, seed):
    errs = _fd_check(opts, nparams, seed)
    fd = np.array([e[1] for e in errs])
    an = np.array([e[2] for e in errs])
    # The FD quotient carries ~5e-8 of FP64 roundoff (the loss sums 196k
    # terms, the step is 1e-6); a 10x larger step is dominated by truncation
    # because the image moves ~70 px per world unit.
    bad = np.abs(fd - an) > 1e-6 * np.abs(an) + 1e-7
    assert not bad.any(), [e for e, b in zip(errs, bad) if b]
    assert np.count_nonzero(np.abs(an) > 1e-4) >= nparams // 2
