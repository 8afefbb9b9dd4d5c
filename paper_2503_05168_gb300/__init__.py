"""GB300 (sm_103a) implementation of the Seele rendering hot path (arxiv 2503.05168).

Thin Python binding over the C ABI in ``include/seele.h``: every step of the
path runs in the CUDA kernels of ``libseele.so``; this module only marshals
arguments.  PyTorch supplies device memory and the stream.

    from paper_2503_05168_gb300 import Renderer
    r = Renderer()
    r.load_scene(scene)            # dict of arrays (numpy: host, torch: device)
    r.set_cameras(cameras)         # list of dicts (world_to_cam, fx, fy, cx, cy, width, height)
    img = r.render(mode="cr")      # flat planar float32 CUDA tensor, all cameras
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import SeeleError, lib

__all__ = ["Renderer", "SeeleError", "SeeleRender", "render", "lib", "default_options", "build", "measure_peaks",
           "exclusive_scan"]


def build(force: bool = False) -> str:
    from .builder import build as _b
    return _b(force=force)


def default_options() -> _abi.Options:
    o = _abi.Options()
    lib().seele_default_options(ctypes.byref(o))
    return o


_CUDART = None


def _cudart():
    """The CUDA runtime already loaded by torch (used for debug copies only)."""
    global _CUDART
    if _CUDART is None:
        for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                _CUDART = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _CUDART is None:
            raise RuntimeError("CUDA runtime library not found")
        _CUDART.cudaMemcpy.restype = ctypes.c_int
        _CUDART.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    return _CUDART


def _ptr(x):
    """Data pointer of a numpy array or torch tensor (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Renderer:
    """One library context on one CUDA device.  Calls enqueue on ``stream``
    (a torch.cuda.Stream) if given, else on the current stream at each call."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.init()
        self._stream = stream
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = lib().seele_create(ctypes.byref(h), device, ctypes.c_void_p(s.cuda_stream))
        if st != 0:
            raise SeeleError(st, "seele_create failed")
        self._h = h
        self._keep = []
        self.cameras = []
        self.n = 0
        self.sh_degree = 0
        self.last_stats = None

    # -- plumbing -----------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise SeeleError(st, lib().seele_last_error(self._h).decode(errors="replace"))

    def _stream_now(self):
        return self._stream if self._stream is not None else self._torch.cuda.current_stream(self.device)

    def _sync_stream(self):
        s = self._stream_now().cuda_stream
        self._check(lib().seele_set_stream(self._h, ctypes.c_void_p(s)))

    def close(self):
        if getattr(self, "_h", None):
            lib().seele_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- scene and cameras ----------------------------------------------------
    def load_scene(self, scene: dict, borrow: bool = False, streamed_slots: int = 0, slot_gaussians: int = 0,
                   ahead: int = 1, spatial: bool = False):
        """``scene``: means [n,3], log_scales [n,3], quats [n,4], opacity_logits [n],
        sh [n,nc,3] (float32), sh_degree, optional cluster_mask [n] uint32,
        centroids [C,6], pos_scale.  numpy arrays are host memory, torch CUDA
        tensors device memory.  ``borrow`` keeps references instead of copying
        (device tensors only).  ``streamed_slots`` > 0 loads a streamed scene
        (seele_load_scene_streamed: host arrays with view clusters; the shared
        Gaussians and that many slots of ``slot_gaussians`` (0: the largest
        cluster) resident, prefetching ``ahead`` frames).  ``spatial`` stores
        the Gaussians in Morton order of their means (SEELE_SCENE_SPATIAL)."""
        torch = self._torch

        def prep(a, dtype):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return a.contiguous() if a.dtype == dtype else a.to(dtype).contiguous()
            return np.ascontiguousarray(a, dtype=np.float32 if dtype == torch.float32 else np.uint32)

        arrs = {k: prep(scene.get(k), torch.float32) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        mask = None
        m = scene.get("cluster_mask")
        if m is not None:
            mask = m.contiguous() if isinstance(m, torch.Tensor) else np.ascontiguousarray(m, dtype=np.uint32)
        cen = scene.get("centroids")
        cen = None if cen is None else np.ascontiguousarray(cen, dtype=np.float32)
        n = int(arrs["means"].shape[0])
        d = _abi.SceneDesc()
        d.n = n
        d.sh_degree = int(scene["sh_degree"])
        d.flags = (_abi.SCENE_BORROW if borrow else _abi.SCENE_COPY) | (_abi.SCENE_SPATIAL if spatial else 0)
        d.means, d.log_scales, d.quats = _ptr(arrs["means"]), _ptr(arrs["log_scales"]), _ptr(arrs["quats"])
        d.opacity_logits, d.sh = _ptr(arrs["opacity_logits"]), _ptr(arrs["sh"])
        d.cluster_mask = _ptr(mask)
        d.n_clusters = 0 if cen is None else int(cen.shape[0])
        d.pos_scale = float(scene.get("pos_scale", 1.0))
        d.centroids = _ptr(cen)
        self._sync_stream()
        if streamed_slots > 0:
            self._check(lib().seele_load_scene_streamed(self._h, ctypes.byref(d), int(streamed_slots),
                                                        int(slot_gaussians), int(ahead)))
        else:
            self._check(lib().seele_load_scene(self._h, ctypes.byref(d)))
        self._keep = [arrs, mask, cen] if borrow else []
        self.n = n
        self.sh_degree = d.sh_degree

    def share_scene(self, other: "Renderer"):
        """Renders ``other``'s scene without a copy (seele_share_scene); this
        renderer keeps its own stream, cameras and frame workspace, so frames
        of both can be in flight at once."""
        self._sync_stream()
        self._check(lib().seele_share_scene(self._h, other._h))
        self._keep = list(other._keep)
        self.n = other.n
        self.sh_degree = other.sh_degree

    @staticmethod
    def _camera_array(cams):
        arr = (_abi.Camera * len(cams))()
        for i, c in enumerate(cams):
            w2c = np.asarray(c["world_to_cam"], dtype=np.float64).reshape(3, 4)
            arr[i].world_to_cam[:] = [float(v) for v in w2c.reshape(-1)]
            arr[i].fx, arr[i].fy = float(c["fx"]), float(c["fy"])
            arr[i].cx, arr[i].cy = float(c["cx"]), float(c["cy"])
            arr[i].width, arr[i].height = int(c["width"]), int(c["height"])
            arr[i].near_z = float(c.get("near", 0.2))
        return arr

    def set_cameras(self, cams):
        arr = self._camera_array(cams)
        self._check(lib().seele_set_cameras(self._h, arr, len(cams)))
        self.cameras = [dict(width=int(c["width"]), height=int(c["height"])) for c in cams]

    @property
    def n_pixels(self):
        return sum(c["width"] * c["height"] for c in self.cameras)

    # -- rendering -----------------------------------------------------------
    @staticmethod
    def make_options(mode="plain", group=(2, 2), tile=(16, 16), opacity_filter=False, cluster_filter=False,
                     n_neighbors=3, sync=True, profile=False, count=False, graph=False, tile_test="ellipse",
                     binning="blocks", schedule="grid", batch_depth=0, **kw) -> _abi.Options:
        o = default_options()
        if tile_test not in ("ellipse", "rect"):
            raise ValueError("tile_test must be 'ellipse' or 'rect'")
        if binning not in ("blocks", "tiles"):
            raise ValueError("binning must be 'blocks' or 'tiles'")
        if schedule not in ("grid", "queue"):
            raise ValueError("schedule must be 'grid' or 'queue'")
        o.schedule = _abi.SCHEDULE_QUEUE if schedule == "queue" else _abi.SCHEDULE_GRID
        o.batch_depth = int(batch_depth)
        o.tile_test = _abi.TILES_ELLIPSE if tile_test == "ellipse" else _abi.TILES_RECT
        o.binning = _abi.BIN_BLOCKS if binning == "blocks" else _abi.BIN_TILES
        o.mode = _abi.MODE_CR if mode == "cr" else _abi.MODE_PLAIN
        o.group_w, o.group_h = group
        o.tile_w, o.tile_h = tile
        o.opacity_filter = int(bool(opacity_filter))
        o.cluster_filter = int(bool(cluster_filter))
        o.n_neighbors = int(n_neighbors)
        for k in ("alpha_min", "alpha_max", "t_stop"):
            if k in kw:
                setattr(o, k, float(kw[k]))
        o.flags = ((0 if sync else _abi.RENDER_ASYNC) | (_abi.RENDER_PROFILE if profile else 0) |
                   (_abi.RENDER_COUNT if count else 0) | (_abi.RENDER_GRAPH if graph else 0))
        return o

    def render(self, out=None, out_T=None, options: _abi.Options | None = None, **kw):
        """Renders every camera; returns the flat planar RGB buffer (``out`` if given).

        ``out``/``out_T`` may be CUDA tensors or host (numpy / CPU torch) buffers."""
        torch = self._torch
        o = options if options is not None else self.make_options(**kw)
        if out is None:
            out = torch.empty(3 * self.n_pixels, dtype=torch.float32, device=self.device)
        st = _abi.Stats()
        self._sync_stream()
        self._check(lib().seele_render(self._h, ctypes.byref(o), ctypes.c_void_p(_ptr(out)),
                                       ctypes.c_void_p(_ptr(out_T)) if out_T is not None else None,
                                       ctypes.byref(st)))
        self.last_stats = dict(n_visible=st.n_visible, n_instances=st.n_instances, capacity=st.capacity,
                               retries=st.retries, n_kernels=st.n_kernels,
                               stage_ms=dict(zip(_abi.STAGES, list(st.stage_ms))),
                               leader_tests=st.leader_tests, pairs_evaluated=st.pairs_evaluated,
                               pairs_blended=st.pairs_blended)
        return out

    def synchronize(self):
        self._check(lib().seele_synchronize(self._h))

    def view_times(self):
        """Per-camera ms from the start of preprocessing to the view's last tile."""
        n = len(self.cameras)
        arr = (ctypes.c_float * n)()
        self._check(lib().seele_get_view_times(self._h, arr, n))
        return list(arr)

    def autotune(self, options: _abi.Options | None = None, **kw):
        """Fastest tile shape for the current scene and cameras: (options, ms)."""
        o = options if options is not None else self.make_options(**kw)
        ms = ctypes.c_float()
        self._sync_stream()
        self._check(lib().seele_autotune(self._h, ctypes.byref(o), ctypes.byref(ms)))
        return o, ms.value

    def autotune_ex(self, objective: str = "batch", cache: str | None = None,
                    options: _abi.Options | None = None, **kw):
        """seele_autotune_ex: tile shape, then schedule and batch depth for
        ``objective`` ("batch", "p50" or "p99"), through the JSON ``cache``
        file if given.  Returns (options, result dict)."""
        objs = {"batch": _abi.TUNE_BATCH_MS, "p50": _abi.TUNE_VIEW_P50, "p99": _abi.TUNE_VIEW_P99}
        o = options if options is not None else self.make_options(**kw)
        res = _abi.TuneResult()
        self._sync_stream()
        self._check(lib().seele_autotune_ex(self._h, ctypes.byref(o), objs[objective],
                                            None if cache is None else str(cache).encode(), ctypes.byref(res)))
        return o, {f: getattr(res, f) for f, _ in _abi.TuneResult._fields_}

    def render_backward(self, dL_drgb) -> dict:
        """Gradients of sum(dL_drgb * rgb) for the last render (CUDA tensors in
        the scene layout): means, log_scales, quats, opacity_logits, sh."""
        torch = self._torch
        dL = dL_drgb.contiguous().to(torch.float32)
        nc = (self.sh_degree + 1) ** 2
        n = self.n
        out = dict(means=torch.empty(n, 3, device=self.device), log_scales=torch.empty(n, 3, device=self.device),
                   quats=torch.empty(n, 4, device=self.device), opacity_logits=torch.empty(n, device=self.device),
                   sh=torch.empty(n, nc, 3, device=self.device))
        G = _abi.Grads(out["means"].data_ptr(), out["log_scales"].data_ptr(), out["quats"].data_ptr(),
                       out["opacity_logits"].data_ptr(), out["sh"].data_ptr())
        self._sync_stream()
        self._check(lib().seele_render_backward(self._h, ctypes.c_void_p(dL.data_ptr()), ctypes.byref(G)))
        return out

    def images(self, flat):
        """Splits a flat planar buffer into per-camera [3, H, W] views."""
        res, off = [], 0
        for c in self.cameras:
            k = 3 * c["width"] * c["height"]
            res.append(flat[off:off + k].reshape(3, c["height"], c["width"]))
            off += k
        return res

    def build_view_clusters(self, poses, n_clusters: int = 16, top_k: int = 32, uniforms=None, seed: int = 0,
                            max_iter: int = 100):
        """Offline view-dependent representation of the loaded scene (Sec. 3.3):
        k-means of the poses on (x / s, v) and per-Gaussian cluster bits from the
        per-pixel top-k contributors.  ``uniforms`` drive k-means++ (default:
        ``n_clusters`` draws of numpy's PCG64 with ``seed``).  Returns
        dict(mask uint32 [n], centroids [C, 6], pos_scale, assign [n_poses])."""
        if uniforms is None:
            uniforms = np.random.default_rng(seed).random(n_clusters)
        u = np.ascontiguousarray(uniforms, np.float64)
        cams = self._camera_array(poses)
        cent = np.zeros((n_clusters, 6), np.float32)
        scale = ctypes.c_float()
        mask = np.zeros(self.n, np.uint32)
        assign = np.zeros(len(poses), np.int32)
        self._sync_stream()
        self._check(lib().seele_build_view_clusters(
            self._h, cams, len(poses), int(n_clusters), int(top_k), ctypes.c_void_p(u.ctypes.data), int(max_iter),
            ctypes.c_void_p(cent.ctypes.data), ctypes.byref(scale), ctypes.c_void_p(mask.ctypes.data),
            ctypes.c_void_p(assign.ctypes.data)))
        return dict(mask=mask, centroids=cent, pos_scale=float(scale.value), assign=assign)

    def stream_stats(self) -> dict:
        """Residency and prefetch counters of a streamed scene."""
        st = _abi.StreamStats()
        self._check(lib().seele_get_stream_stats(self._h, ctypes.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in _abi.StreamStats._fields_}

    def contribution_skew(self, frac: float = 0.99, tile=(16, 16), tile_test="ellipse", **kw):
        """Contribution skew of a plain render of the current cameras (Sec. 1,
        Sec. 3.4): per camera, dict(m, blended, walked, total, listed) as
        [H, W] numpy arrays -- m the smallest number of a pixel's largest
        contributions Gamma alpha that sum to ``frac`` of their total, listed
        the length of its tile list."""
        o = self.make_options(mode="plain", tile=tile, tile_test=tile_test, binning="tiles", **kw)
        P = self.n_pixels
        m = np.zeros(P, np.uint32)
        blended = np.zeros(P, np.uint32)
        walked = np.zeros(P, np.uint32)
        total = np.zeros(P, np.float32)
        listed = np.zeros(P, np.uint32)
        self._sync_stream()
        self._check(lib().seele_contribution_skew(
            self._h, ctypes.byref(o), ctypes.c_float(frac), ctypes.c_void_p(m.ctypes.data),
            ctypes.c_void_p(blended.ctypes.data), ctypes.c_void_p(walked.ctypes.data),
            ctypes.c_void_p(total.ctypes.data), ctypes.c_void_p(listed.ctypes.data)))
        out, off = [], 0
        for c in self.cameras:
            W, H = c["width"], c["height"]
            sl = slice(off, off + W * H)
            out.append(dict(m=m[sl].reshape(H, W), blended=blended[sl].reshape(H, W),
                            walked=walked[sl].reshape(H, W), total=total[sl].reshape(H, W),
                            listed=listed[sl].reshape(H, W)))
            off += W * H
        return out

    def debug_view(self) -> dict:
        """Copies of the last render's intermediates (CUDA tensors)."""
        torch = self._torch
        v = _abi.DebugView()
        self._check(lib().seele_get_debug_view(self._h, ctypes.byref(v)))

        def dev(ptr, count, dtype):
            if count == 0:
                return torch.empty(0, dtype=dtype, device=self.device)
            out = torch.empty(count, dtype=dtype, device=self.device)
            self._stream_now().synchronize()
            res = _cudart().cudaMemcpy(ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ptr),
                                       ctypes.c_size_t(count * out.element_size()), 3)  # device to device
            if int(res) != 0:
                raise RuntimeError(f"cudaMemcpy failed: {res}")
            return out

        R, K, T = v.n_records, v.n_instances, v.n_tiles
        i32 = torch.int32
        start = dev(v.tile_start, T, i32).to(torch.int64) & 0xFFFFFFFF   # stored as uint32
        end = dev(v.tile_end, T, i32).to(torch.int64)
        empty = start >= end
        ranges = torch.stack([torch.where(empty, 0, start), torch.where(empty, 0, end)], 1).to(i32)
        counts = (ranges[:, 1] - ranges[:, 0]).to(torch.int64)
        inst_tile = torch.repeat_interleave(torch.arange(T, device=self.device, dtype=i32), counts)
        records = dev(v.records, 16 * R, torch.float32).reshape(R, 16)
        return dict(
            n_records=R, n_visible=v.n_visible, n_instances=K, n_tiles=T,
            inst_tile=inst_tile, inst_record=dev(v.inst_record, K, i32),
            tile_ranges=ranges,
            tiles_touched=dev(v.tiles_touched, R, i32), rect=records[:, 12:14].contiguous().view(i32),
            records=records[:, :12].contiguous(), depth=dev(v.depth, R, torch.float32),
            n_contrib=dev(v.n_contrib, self.n_pixels, i32),
            inst_mask=dev(v.inst_mask, K, i32) if v.inst_mask else None,
            scene_order=dev(v.scene_order, R // max(1, len(self.cameras)), i32) if v.scene_order else None,
            mask_summary=dev(v.mask_summary, (K + 31) // 32, i32) if v.mask_summary else None,
        )


def _autograd_function():
    import torch

    class SeeleRender(torch.autograd.Function):
        """Differentiable render: the forward pass borrows the attribute tensors
        (no copy) and renders every camera of ``renderer``; the backward pass
        runs the library's backward kernels.  One render per renderer may be
        awaiting its backward at a time."""

        @staticmethod
        def forward(ctx, renderer, options, sh_degree, means, log_scales, quats, opacity_logits, sh):
            renderer.load_scene(dict(means=means, log_scales=log_scales, quats=quats,
                                     opacity_logits=opacity_logits, sh=sh, sh_degree=sh_degree), borrow=True)
            img = renderer.render(options=options)
            ctx.renderer = renderer
            return img

        @staticmethod
        def backward(ctx, grad_img):
            g = ctx.renderer.render_backward(grad_img)
            return None, None, None, g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"]

    return SeeleRender


class _Lazy:
    fn = None


def __getattr__(name):
    if name == "SeeleRender":
        if _Lazy.fn is None:
            _Lazy.fn = _autograd_function()
        return _Lazy.fn
    raise AttributeError(name)


def render(renderer: "Renderer", means, log_scales, quats, opacity_logits, sh, sh_degree: int = 3, **options):
    """Differentiable render of every camera of ``renderer`` (flat planar RGB).
    Bins by tiles unless told otherwise: the backward pass walks tile lists."""
    fn = __getattr__("SeeleRender")
    options.setdefault("binning", "tiles")
    o = renderer.make_options(**options)
    return fn.apply(renderer, o, sh_degree, means, log_scales, quats, opacity_logits, sh)


def measure_peaks(device: int = 0) -> dict:
    """seele_measure_peaks: measured FP32 (FMA), SFU (ex2) and ALU (float
    min/max, integer logic) lane-op rates of ``device`` in 1e12 per second,
    its SM count and maximum SM clock (MHz), on the current stream."""
    import torch
    s = torch.cuda.current_stream(torch.device("cuda", device)).cuda_stream
    p = _abi.Peaks()
    st = lib().seele_measure_peaks(device, ctypes.c_void_p(s), ctypes.byref(p))
    if st != 0:
        raise SeeleError(st, "seele_measure_peaks failed")
    return {f: getattr(p, f) for f, _ in _abi.Peaks._fields_}


def exclusive_scan(x, withhold_block: int | None = None, spin_limit: int = 0):
    """seele_exclusive_scan of a 1-D int32/uint32 CUDA tensor (16-byte
    aligned); returns (status, out).  ``withhold_block`` and ``spin_limit`` are
    the call's test hook for the bounded look-back wait."""
    import torch
    n = int(x.numel())
    out = torch.empty_like(x)
    scratch = torch.empty(int(lib().seele_scan_scratch_bytes(n)) + 256, dtype=torch.uint8, device=x.device)
    base = (scratch.data_ptr() + 255) // 256 * 256
    s = torch.cuda.current_stream(x.device).cuda_stream
    st = lib().seele_exclusive_scan(ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(base), 0xFFFFFFFF if withhold_block is None else withhold_block,
                                    spin_limit, ctypes.c_void_p(s))
    return st, out
