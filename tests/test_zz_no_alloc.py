"""usv_insert_pnn_noalloc, the insertion entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library),
checked through the C ABI against the regular entry point: the packed
accumulators must be bit-identical after each of two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from helpers import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def _entry():
    from paper_2412_00058_gb300 import usvol
    f = usvol.lib().usv_insert_pnn_noalloc
    D3 = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [ctypes.c_void_p, usvol.Grid, D3, D3, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.POINTER(usvol.Calibration), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_insert_matches_regular_insert_on_two_calls_in_a_row():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.whole_spine(n=30, grid=(270, 70, 200), y_start_mm=4.0, y_span_mm=10.0)
    nx, ny, nz = w.grid
    f = _entry()
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    cal = usvol.calibration_of(w)
    stream = usvol._stream_ptr(None)
    acc = torch.zeros((nz, ny, nx), dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    vol.reset()
    for a, b, st in [(0, 17, status), (17, 30, None)]:     # two calls in a row
        rc = f(acc.data_ptr(), usvol.Grid(nx, ny, nz), usvol._d3(w.spacing),
               usvol._d3(w.origin), imgs[a:b].data_ptr(), b - a, w.H, w.W,
               poses[a:b].data_ptr(), ctypes.byref(cal),
               st.data_ptr() if st is not None else None, stream)
        assert rc == usvol.OK, usvol.strerror(rc)
        vol.insert(imgs[a:b], poses[a:b], cal)
        ref = vol.read(usvol.READ_ACCUM)
        torch.cuda.synchronize()
        assert torch.equal(acc, ref), f"accumulators differ after frames [{a},{b})"
    assert int(status.item()) == 0
    assert int((acc >> 32).sum().item()) > 0


def test_noalloc_reports_bad_poses_and_rejects_oversized_batches():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=6, H=32, W=32, grid=(40, 40, 40), sweep_mm=5.0, y0_mm=3.0)
    w.poses[2, 0, 3] = np.nan
    nx, ny, nz = w.grid
    f = _entry()
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    cal = usvol.calibration_of(w)
    stream = usvol._stream_ptr(None)
    acc = torch.zeros((nz, ny, nx), dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (acc.data_ptr(), usvol.Grid(nx, ny, nz), usvol._d3(w.spacing), usvol._d3(w.origin),
            imgs.data_ptr())
    rc = f(*args, 6, w.H, w.W, poses.data_ptr(), ctypes.byref(cal), status.data_ptr(), stream)
    assert rc == usvol.OK
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    vol.reset()
    vol.insert(imgs, poses, cal)
    assert torch.equal(acc, vol.read(usvol.READ_ACCUM))
    torch.cuda.synchronize()
    assert int(status.item()) & usvol.STATUS_BAD_POSE
    rc = f(*args, 1025, w.H, w.W, poses.data_ptr(), ctypes.byref(cal), None, stream)
    assert rc == usvol.ERR_RANGE
