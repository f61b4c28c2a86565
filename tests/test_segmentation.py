"""Tissue segmentation by depth of cut (the paper's Algorithms 1 and 2):
oracle pins on the CPU (closed forms, hand-built frames), GPU parity
through the C ABI (bit-exact rows and nearest-neighbour volumes)."""
import ctypes
import math

import numpy as np
import pytest

import oracle


def rigid(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


# ---------------------------------------------------------------- oracle pins

def test_alg1_cut_depth_closed_form():
    """Cut_n = K |P_c1.x - P_cn.x - L/2| + D with the spine along -y of the
    world (so the distance travelled from the first frame is positive):
    K = 0.5, D = 30 mm, L = 400 mm; frames whose upper-left pixel sits at
    y = 0, 100, 200, 300 mm cut at 130, 80, 30, 80 mm -- shallow in the middle
    of the back, deeper towards the ends (Sec. II.D)."""
    poses = np.stack([rigid(np.eye(3), (5.0, y, 2.0)) for y in (0.0, 100.0, 200.0, 300.0)])
    rows, cut = oracle.cut_rows_alg1(poses, 1000, np.eye(4), 0.5, 30.0, 400.0, (0, -1, 0),
                                     (5.0, 0.0, 2.0), 0.5)
    assert list(cut) == [130.0, 80.0, 30.0, 80.0]
    assert list(rows) == [260, 160, 60, 160]
    rows, _ = oracle.cut_rows_alg1(poses, 100, np.eye(4), 0.5, 30.0, 400.0, (0, -1, 0),
                                   (5.0, 0.0, 2.0), 0.5)
    assert list(rows) == [100, 100, 60, 100]              # clamped to H
    # the calibration moves the upper-left pixel: K shifts the image 10 mm along +y
    K = rigid(np.eye(3), (0.0, 10.0, 0.0))
    _, cut = oracle.cut_rows_alg1(poses[:1], 1000, K, 0.5, 30.0, 400.0, (0, -1, 0),
                                  (5.0, 0.0, 2.0), 0.5)
    assert cut[0] == 0.5 * abs(10.0 - 200.0) + 30.0     # (p1 - pn).e = (-10)(-1)


def _bone_frames(rows, H=64, W=24, drop=2):
    imgs = np.full((len(rows), H, W), 50, np.uint8)
    for f, r in enumerate(rows):
        imgs[f, r, :] = 250
        imgs[f, r + 1:, :] = 10
    return imgs


def test_alg2_bone_row_and_temporal_median():
    imgs = _bone_frames([40, 40, 20, 41, 40])
    bone, rows = oracle.bone_rows_alg2(imgs, 8, 2, 3, 3)
    assert list(bone) == [40, 40, 20, 41, 40]
    # window 3, clipped at the ends: medians of {40,40}, {40,40,20}, {40,20,41},
    # {20,41,40}, {41,40} (lower medians) minus 3
    assert list(rows) == [37, 37, 37, 37, 37]
    bone, rows = oracle.bone_rows_alg2(imgs, 8, 2, 1, 0)
    assert list(rows) == [40, 40, 20, 41, 40]
    # search region excludes a brighter contour above it
    imgs2 = _bone_frames([40])
    imgs2[0, 5, :] = 255
    imgs2[0, 6:40, :] = 0
    bone, _ = oracle.bone_rows_alg2(imgs2, 10, 2, 1, 0)
    assert bone[0] == 40
    bone, _ = oracle.bone_rows_alg2(imgs2, 0, 2, 1, 0)
    assert bone[0] == 5


def test_alg2_lower_median_over_columns():
    imgs = _bone_frames([30], W=5)
    imgs[0, :, 0] = 50          # flat column: no contour -> search start row
    imgs[0, 30:, 1] = 50
    imgs[0, 44, 1] = 250        # column 1: contour at 44
    imgs[0, 45:, 1] = 10
    bone, _ = oracle.bone_rows_alg2(imgs, 8, 2, 1, 0)
    assert bone[0] == 30        # sorted rows 8, 30, 30, 30, 44 -> 3rd


def test_cut_insert_equals_inserting_the_cropped_image():
    """Cutting rows above r equals inserting rows [r, H) as their own image
    whose calibration is shifted r*sy down (exact values, identity pose)."""
    rng = np.random.default_rng(3)
    imgs = rng.integers(0, 256, size=(2, 12, 10), dtype=np.uint8)
    poses = np.stack([rigid(np.eye(3), (0.5, 1.0, 0.0)), rigid(np.eye(3), (1.0, 1.5, 0.5))])
    grid = (16, 6, 14)
    s, c, _ = oracle.insert_pnn(grid, imgs, poses, np.eye(4), 0.5, 0.5, (0.5,) * 3, (0, 0, 0),
                                first_rows=np.array([4, 7]))
    ref_s = np.zeros_like(s)
    ref_c = np.zeros_like(c)
    for f, r in enumerate((4, 7)):
        K = rigid(np.eye(3), (0.0, 0.0, r * 0.5))
        oracle.insert_pnn(grid, imgs[f:f + 1, r:], poses[f:f + 1], K, 0.5, 0.5, (0.5,) * 3,
                          (0, 0, 0), sum_=ref_s, cnt=ref_c)
    assert np.array_equal(s, ref_s) and np.array_equal(c, ref_c)
    assert 0 < c.sum() <= (12 - 4) * 10 + (12 - 7) * 10


# ---------------------------------------------------------------- GPU parity

def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from helpers import build_library
    build_library()


@pytest.mark.gpu
def test_gpu_alg1_rows_and_cut_insert_bit_exact():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    from helpers import assert_pnn_bit_exact, gpu_run
    _gpu()
    w = synth.whole_spine(n=40, grid=(270, 120, 200), y_start_mm=20.0, y_span_mm=30.0)
    p1 = (w.poses[0] @ w.calib)[:3, 3]
    prm = dict(k=0.4, d_mm=25.0, l_mm=40.0, spine_dir=(0.0, -1.0, 0.0))
    rows, _ = oracle.cut_rows_alg1(w.poses, w.H, w.calib, prm["k"], prm["d_mm"], prm["l_mm"],
                                   prm["spine_dir"], p1, w.sy)
    L = usvol.lib()
    a1 = usvol.Alg1Params(prm["k"], prm["d_mm"], prm["l_mm"], (ctypes.c_double * 3)(*prm["spine_dir"]),
              (ctypes.c_double * 3)(*p1))
    poses = torch.from_numpy(w.poses).cuda()
    drows = torch.empty(w.n, dtype=torch.int32, device="cuda")
    cal = usvol.calibration_of(w)
    rc = L.usv_cut_rows_alg1(poses.data_ptr(), w.n, w.H, ctypes.byref(cal), ctypes.byref(a1),
                             drows.data_ptr(), usvol._stream_ptr(None))
    assert rc == 0
    assert np.array_equal(drows.cpu().numpy(), rows)
    assert rows.min() < rows.max()                       # the cut varies along the sweep
    # insert with the cut, against the oracle with the same rows
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    vol.reset()
    imgs = torch.from_numpy(w.images).cuda()
    rc = L.usv_insert_frames_cut(vol.handle, imgs.data_ptr(), w.n, w.H, w.W, usvol.U8,
                                 poses.data_ptr(), ctypes.byref(cal), drows.data_ptr(),
                                 usvol._stream_ptr(None))
    assert rc == 0
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    s, c, _ = oracle.insert_pnn(w.grid, w.images, w.poses, w.calib, w.sx, w.sy, w.spacing,
                                w.origin, first_rows=rows)
    assert np.array_equal(acc & np.uint64(0xFFFFFFFF), s)
    assert np.array_equal(acc >> np.uint64(32), c.astype(np.uint64))


@pytest.mark.gpu
def test_gpu_alg2_rows_bit_exact_on_the_sweep():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    _gpu()
    w = synth.whole_spine(n=60, grid=(270, 200, 200), y_start_mm=10.0, y_span_mm=40.0)
    prm = (w.H // 3, 6, 15, 20)   # search the lower two thirds; shadow 6 rows below
    bone, rows = oracle.bone_rows_alg2(w.images, *prm)
    L = usvol.lib()
    Alg2 = usvol.Alg2Params
    imgs = torch.from_numpy(w.images).cuda()
    db = torch.empty(w.n, dtype=torch.int32, device="cuda")
    dr = torch.empty(w.n, dtype=torch.int32, device="cuda")
    rc = L.usv_bone_rows_alg2(imgs.data_ptr(), w.n, w.H, w.W, ctypes.byref(Alg2(*prm)),
                              db.data_ptr(), dr.data_ptr(), usvol._stream_ptr(None))
    assert rc == 0
    assert np.array_equal(db.cpu().numpy(), bone) and np.array_equal(dr.cpu().numpy(), rows)
    # the synthetic bone arc sits at depth 45 + 15 sin(2 pi y / 550) mm minus a
    # 4 mm lateral curvature: the detected row is within the arc's depth range
    depth = 45.0 + 15.0 * np.sin(2 * np.pi * w.poses[:, 1, 3] / 550.0)
    assert np.all(np.abs(bone * w.sy - (depth - 4 * (2 / 3))) < 4.0)
    assert L.usv_bone_rows_alg2(imgs.data_ptr(), w.n, w.H, w.W,
                                ctypes.byref(Alg2(0, 6, 4, 0)), db.data_ptr(), dr.data_ptr(),
                                usvol._stream_ptr(None)) == usvol.ERR_ARG   # even window
