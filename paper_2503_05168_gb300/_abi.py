"""ctypes mirror of include/seele.h (structs, enums, prototypes).

Loading fails loudly when libseele.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SEELE_LIBRARY selects another build of the same ABI (the checked build)
LIB_PATH = os.environ.get("SEELE_LIBRARY") or os.path.join(HERE, "libseele.so")

SEELE_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_CUDA", 4: "ERR_CAPACITY", 5: "ERR_TIMEOUT",
                6: "ERR_OOM", 7: "ERR_INTERNAL"}
SCENE_COPY, SCENE_BORROW, SCENE_SPATIAL = 0, 1, 2
MODE_PLAIN, MODE_CR = 0, 1
TILES_RECT, TILES_ELLIPSE = 0, 1
BIN_TILES, BIN_BLOCKS = 0, 1
SCHEDULE_GRID, SCHEDULE_QUEUE = 0, 1
TUNE_BATCH_MS, TUNE_VIEW_P50, TUNE_VIEW_P99 = 0, 1, 2
RENDER_ASYNC = 1
RENDER_PROFILE = 2
RENDER_COUNT = 4
RENDER_GRAPH = 8
STAGES = ("preprocess", "compact", "depth_sort", "tile_scan", "emit", "tile_sort", "ranges", "raster")

P = ctypes.c_void_p


class SceneDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("means", P), ("log_scales", P), ("quats", P), ("opacity_logits", P), ("sh", P),
                ("cluster_mask", P), ("n_clusters", ctypes.c_int32), ("pos_scale", ctypes.c_float),
                ("centroids", P)]


class Camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_z", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("group_w", ctypes.c_int32), ("group_h", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("opacity_filter", ctypes.c_int32),
                ("cluster_filter", ctypes.c_int32), ("n_neighbors", ctypes.c_int32),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float), ("t_stop", ctypes.c_float),
                ("flags", ctypes.c_int32), ("tile_test", ctypes.c_int32), ("binning", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("batch_depth", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_int64), ("n_instances", ctypes.c_int64), ("capacity", ctypes.c_int64),
                ("retries", ctypes.c_int32), ("n_kernels", ctypes.c_int32), ("stage_ms", ctypes.c_float * 8),
                ("leader_tests", ctypes.c_int64), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_blended", ctypes.c_int64)]


class StreamStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("resident_bytes", "full_bytes", "n_shared", "slot_capacity", "n_slots",
                                              "n_chunks", "frames", "loads_sync", "loads_prefetched",
                                              "prefetch_hits", "resident_hits")]


class TuneResult(ctypes.Structure):
    _fields_ = [("batch_ms", ctypes.c_float), ("view_p50_ms", ctypes.c_float), ("view_p99_ms", ctypes.c_float),
                ("from_cache", ctypes.c_int32), ("candidates", ctypes.c_int32)]


class Peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("sm_clock_max_mhz", ctypes.c_int32), ("fp32_tops", ctypes.c_double),
                ("sfu_tops", ctypes.c_double), ("alu_fmnmx_tops", ctypes.c_double),
                ("alu_lop3_tops", ctypes.c_double), ("fp32_ms", ctypes.c_float), ("sfu_ms", ctypes.c_float),
                ("alu_fmnmx_ms", ctypes.c_float), ("alu_lop3_ms", ctypes.c_float)]


class Grads(ctypes.Structure):
    _fields_ = [("means", P), ("log_scales", P), ("quats", P), ("opacity_logits", P), ("sh", P)]


class DebugView(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_int64), ("n_visible", ctypes.c_int64), ("n_instances", ctypes.c_int64),
                ("n_tiles", ctypes.c_int64), ("inst_record", P), ("tile_start", P), ("tile_end", P),
                ("tiles_touched", P), ("records", P), ("depth", P), ("n_contrib", P),
                ("inst_mask", P), ("scene_order", P), ("mask_summary", P)]


# name -> (restype, argtypes); the ABI test checks this table against the header
PROTOTYPES = {
    "seele_default_options": (None, [ctypes.POINTER(Options)]),
    "seele_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
    "seele_destroy": (None, [P]),
    "seele_set_stream": (ctypes.c_int, [P, P]),
    "seele_load_scene": (ctypes.c_int, [P, ctypes.POINTER(SceneDesc)]),
    "seele_set_cameras": (ctypes.c_int, [P, ctypes.POINTER(Camera), ctypes.c_int32]),
    "seele_render": (ctypes.c_int, [P, ctypes.POINTER(Options), P, P, ctypes.POINTER(Stats)]),
    "seele_synchronize": (ctypes.c_int, [P]),
    "seele_render_backward": (ctypes.c_int, [P, P, ctypes.POINTER(Grads)]),
    "seele_get_debug_view": (ctypes.c_int, [P, ctypes.POINTER(DebugView)]),
    "seele_last_error": (ctypes.c_char_p, [P]),
    "seele_get_view_times": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "seele_autotune": (ctypes.c_int, [P, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_float)]),
    "seele_autotune_ex": (ctypes.c_int, [P, ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_char_p,
                                         ctypes.POINTER(TuneResult)]),
    "seele_sort_tile_instances_noalloc": (ctypes.c_int, [P, P, ctypes.c_uint32, ctypes.c_uint32, P, P, P, P]),
    "seele_build_view_clusters": (ctypes.c_int, [P, ctypes.POINTER(Camera), ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, P, ctypes.c_int32, P, P, P, P]),
    "seele_contribution_skew": (ctypes.c_int, [P, ctypes.POINTER(Options), ctypes.c_float, P, P, P, P, P]),
    "seele_load_scene_streamed": (ctypes.c_int, [P, ctypes.POINTER(SceneDesc), ctypes.c_int32, ctypes.c_int64,
                                                 ctypes.c_int32]),
    "seele_get_stream_stats": (ctypes.c_int, [P, ctypes.POINTER(StreamStats)]),
    "seele_share_scene": (ctypes.c_int, [P, P]),
    "seele_measure_peaks": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(Peaks)]),
    "seele_scan_scratch_bytes": (ctypes.c_size_t, [ctypes.c_uint32]),
    "seele_exclusive_scan": (ctypes.c_int, [P, ctypes.c_uint32, P, P, ctypes.c_uint32, ctypes.c_uint32, P]),
}
NOALLOC_MAX_INSTANCES = 1 << 20
NOALLOC_MAX_TILES = 1 << 16

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2503_05168_gb300.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SeeleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
