"""The C-ABI library builds, loads and exports every symbol include/usvol.h
declares; host-side argument checks reject bad input before any CUDA call
(CPU only: no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def usvol():
    from paper_2412_00058_gb300 import build, usvol
    build.build()
    usvol.lib()
    return usvol


def header_functions():
    text = open(os.path.join(ROOT, "include", "usvol.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(usv_\w+)\s*\(", text))


def test_header_symbols_exported(usvol):
    names = header_functions()
    assert names == set(usvol.EXPORTS)
    L = usvol.lib()
    for n in names:
        assert hasattr(L, n), f"{n} not exported by libusvol.so"
    assert L.usv_abi_version() == 2


def test_library_is_sm103a_build(usvol):
    from paper_2412_00058_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_volume_bytes(usvol):
    assert usvol.volume_bytes((0, 4, 4), usvol.PNN) == 0
    assert usvol.volume_bytes((4, 4, 4), 7) == 0
    assert usvol.volume_bytes((2 ** 11, 2 ** 10, 2 ** 10), usvol.PNN) == 0   # > 2^31-1 voxels
    n = 270 * 1840 * 200
    b = usvol.volume_bytes((270, 1840, 200), usvol.PNN)
    assert n * 9.125 < b < n * 9.125 + 4 * 2 ** 20
    bt = usvol.volume_bytes((270, 1840, 200), usvol.TRILINEAR)
    assert n * 12.125 < bt < n * 12.125 + 4 * 2 ** 20


def test_create_rejects_bad_arguments_on_host(usvol):
    L = usvol.lib()
    h = ctypes.c_void_p()
    G = usvol.Grid
    ok3 = usvol._d3((0.3, 0.3, 0.3))
    o3 = usvol._d3((0, 0, 0))
    big = 1 << 40
    fake = ctypes.c_void_p(1 << 20)          # aligned, never dereferenced
    assert L.usv_volume_create(G(4, 4, 4), ok3, o3, 0, fake, big, None) == usvol.ERR_ARG
    assert L.usv_volume_create(G(0, 4, 4), ok3, o3, 0, fake, big, ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), usvol._d3((0.3, 0, 0.3)), o3, 0, fake, big,
                               ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), usvol._d3((0.3, float("nan"), 0.3)), o3, 0, fake, big,
                               ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), ok3, usvol._d3((0, float("inf"), 0)), 0, fake, big,
                               ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), ok3, o3, 3, fake, big, ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), ok3, o3, 0, None, big, ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), ok3, o3, 0, ctypes.c_void_p((1 << 20) + 8), big,
                               ctypes.byref(h)) == usvol.ERR_ARG
    assert L.usv_volume_create(G(4, 4, 4), ok3, o3, 0, fake, 100, ctypes.byref(h)) == usvol.ERR_NOMEM
    assert h.value is None


def test_calls_on_null_handle_fail_cleanly(usvol):
    L = usvol.lib()
    cal = usvol.make_calibration([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1], sx=0.3, sy=0.3)
    assert L.usv_insert_frames(None, None, 1, 4, 4, 0, None, ctypes.byref(cal), None) == usvol.ERR_ARG
    assert L.usv_insert_frames_dev(None, None, 1, 4, 4, 0, None, ctypes.byref(cal),
                                   None) == usvol.ERR_ARG
    assert L.usv_test_insert_trilinear_carry(None, None, 1, 4, 4, 0, None, ctypes.byref(cal), 1,
                                             None) == usvol.ERR_ARG
    assert L.usv_fill_holes(None, 1, None) == usvol.ERR_ARG
    assert L.usv_project_depth_band(None, 0, 1, None, None, None) == usvol.ERR_ARG
    assert L.usv_volume_read(None, 0, None, None) == usvol.ERR_ARG
    assert L.usv_volume_reset(None, None) == usvol.ERR_ARG
    assert L.usv_status(None, None) == usvol.ERR_ARG
    assert L.usv_volume_destroy(None) == usvol.ERR_ARG
    assert usvol.strerror(usvol.ERR_NOMEM).startswith("device storage")
    assert usvol.strerror(12345) == "unknown usvol error"


def test_volume_bytes_with_spare_accumulators(usvol):
    n = 270 * 1840 * 200
    b = usvol.volume_bytes((270, 1840, 200), usvol.PNN)
    bs = usvol.volume_bytes((270, 1840, 200), usvol.PNN | usvol.SPARE_ACCUM)
    assert bs - b == (n * 8 + 255) // 256 * 256
    bt = usvol.volume_bytes((40, 30, 20), usvol.TRILINEAR | usvol.SPARE_ACCUM)
    assert bt - usvol.volume_bytes((40, 30, 20), usvol.TRILINEAR) == 40 * 30 * 20 * 8
    assert usvol.volume_bytes((4, 4, 4), 0x200) == 0
    assert usvol.volume_bytes((4, 4, 4), usvol.SPARE_ACCUM | 2) == 0


def test_new_calls_reject_bad_arguments_on_host(usvol):
    L = usvol.lib()
    cfg = usvol.TileConfig(128, 64, 8)
    assert L.usv_fill_holes_and_clear(None, 1, None) == usvol.ERR_ARG
    assert L.usv_set_tile_config(None, 4, 4, ctypes.byref(cfg)) == usvol.ERR_ARG
    assert L.usv_get_tile_config(None, 4, 4, ctypes.byref(cfg)) == usvol.ERR_ARG
    assert L.usv_tune_insert(None, None, 1, 4, 4, 0, None, None, None, ctypes.c_size_t(0),
                             None, None, None) == usvol.ERR_ARG
    # multi-job insertion: the job list is checked before any device work
    assert L.usv_insert_frames_multi(None, 0, None) == usvol.OK
    assert L.usv_insert_frames_multi(None, 1, None) == usvol.ERR_ARG
    assert L.usv_insert_frames_multi(None, -1, None) == usvol.ERR_ARG
    jobs = (usvol.InsertJob * 33)()
    assert L.usv_insert_frames_multi(jobs, 33, None) == usvol.ERR_RANGE
    assert L.usv_insert_frames_multi(jobs, 2, None) == usvol.ERR_ARG   # null volumes
