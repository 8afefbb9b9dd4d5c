"""The C ABI library builds, loads without a GPU, exports every function that
include/seele.h declares, and the ctypes mirror has the header's layouts."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2503_05168_gb300 import _abi
from paper_2503_05168_gb300.builder import build as build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "seele.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(seele_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    path = build_lib()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_abi.PROTOTYPES), set(names) ^ set(_abi.PROTOTYPES)


def test_default_options_are_the_papers_constants(lib):
    o = _abi.Options()
    lib.seele_default_options(ctypes.byref(o))
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and (o.group_w, o.group_h) == (2, 2)
    assert o.mode == _abi.MODE_PLAIN and abs(o.alpha_max - 0.99) < 1e-7 and abs(o.t_stop - 1e-4) < 1e-10
    assert o.tile_test == _abi.TILES_ELLIPSE
    assert o.n_neighbors == 3


def test_create_without_device_is_an_argument_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    lib.seele_create.restype = ctypes.c_int
    assert lib.seele_create(ctypes.byref(h), 0, None) != 0
    assert not h.value


STRUCTS = {
    "seele_scene_desc": _abi.SceneDesc, "seele_camera": _abi.Camera, "seele_options": _abi.Options,
    "seele_stats": _abi.Stats, "seele_grads": _abi.Grads, "seele_debug_view": _abi.DebugView,
    "seele_peaks": _abi.Peaks, "seele_tune_result": _abi.TuneResult,
}


def test_ctypes_layouts_match_the_header():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "seele.h"', "int main(void){"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    got = dict(l.split() for l in out if l.strip())
    for cname, py in STRUCTS.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_argument_checks_come_before_any_gpu_work(lib):
    """Calls that must refuse their arguments do so without touching memory
    or a device (the pointers below are never dereferenced)."""
    L = _abi.lib()
    fake = [ctypes.c_void_p(0x100000 + 0x1000 * i) for i in range(5)]
    # no-alloc sort: the tile ids are read as 16-byte vectors
    mis = ctypes.c_void_p(0x100004)
    assert L.seele_sort_tile_instances_noalloc(mis, fake[1], 8, 4, fake[2], fake[3], fake[4], None) == 1
    assert L.seele_sort_tile_instances_noalloc(fake[0], fake[1], 8, 4, fake[2], None, fake[4], None) == 1
    # scan: misaligned scratch or input, NULL pointers
    assert L.seele_exclusive_scan(fake[0], 8, fake[1], ctypes.c_void_p(0x100010), 0xFFFFFFFF, 0, None) == 1
    assert L.seele_exclusive_scan(mis, 8, fake[1], fake[2], 0xFFFFFFFF, 0, None) == 1
    assert L.seele_exclusive_scan(None, 8, fake[1], fake[2], 0xFFFFFFFF, 0, None) == 1
    assert L.seele_measure_peaks(0, None, None) == 1
    assert L.seele_scan_scratch_bytes(4096 * 16) == 256 + 8 * 16
