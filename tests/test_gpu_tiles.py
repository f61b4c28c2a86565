"""Insertion tile shapes and the autotuner, through the C ABI: every tile
shape gives bit-exact nearest-neighbour volumes (the result cannot depend on
how frames are cut into tiles) and trilinear volumes within the FP64
oracle's tolerance; the autotuner keeps a valid shape per frame size."""
import numpy as np
import pytest

from helpers import assert_pnn_bit_exact, assert_trilinear_close, build_library, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def run_with_tile(w, cfg, tune=False):
    """Insert, fill and project w with a given tile shape (or the tuned one)."""
    import torch
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume(w.grid, w.spacing, w.origin, w.mode)
    imgs = torch.from_numpy(np.ascontiguousarray(w.images)).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses)).cuda()
    cal = usvol.calibration_of(w)
    n, H, W = w.images.shape
    tuned = None
    if tune:
        tuned = vol.tune(imgs, poses, cal)
        assert vol.get_tile(H, W) == tuned[0]
    elif cfg is not None:
        vol.set_tile(H, W, cfg)
        assert vol.get_tile(H, W) == tuple(cfg)
    vol.reset()
    vol.insert(imgs, poses, cal)
    vol.fill()
    lo, hi = w.band
    out, cnt = vol.project(lo, hi)
    res = dict(status=vol.status(), band=(lo, hi), tuned=tuned, vol=vol)
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy()
    if w.mode == "pnn":
        acc = acc.view(np.uint64)
        res["sum"] = acc & np.uint64(0xFFFFFFFF)
        res["cnt"] = (acc >> np.uint64(32)).astype(np.uint32)
    else:
        res["S"], res["W"] = acc[..., 0].astype(np.float64), acc[..., 1].astype(np.float64)
    res["val"] = vol.read(usvol.READ_VALUES).cpu().numpy()
    res["has"] = vol.read(usvol.READ_MASK).cpu().numpy()
    res["proj"] = out.cpu().numpy()
    res["pcnt"] = cnt.cpu().numpy().view(np.uint16)
    return res


PNN_SHAPES = [(tw, th, f) for tw in (64, 128, 256) for th in (32, 48, 64, 96, 128)
              for f in (4, 8, 12, 16) if tw < 256 or f <= 8]
PNN_SHAPES += [(128, 7, 3), (64, 1, 1), (256, 200, 8), (64, 640, 2), (128, 64, 6),
               (128, 64, 11), (64, 5, 13)]


def test_every_pnn_tile_shape_bit_exact():
    """Whole-spine geometry (480x640 frames, in-plane tilt) with every tile
    shape the autotuner tries plus ragged ones (7-row tiles, single rows,
    tiles taller than the frame, 3 frames per block)."""
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=21, grid=(270, 60, 200), y_start_mm=3.0, y_span_mm=8.0)
    o = oracle_run(w)
    for cfg in PNN_SHAPES:
        g = run_with_tile(w, cfg)
        assert g["status"] == 0
        assert_pnn_bit_exact(g, o)


@pytest.mark.parametrize("span_mm", [8.0, 14.0])
def test_pnn_two_pass_groups_bit_exact(span_mm):
    """Frames about one voxel apart (14 mm over 48 frames) make the box of
    12 or 16 frames too large for packed shared-memory entries in most
    tiles, so those blocks insert their group as two passes (the first 8
    frames, then the rest), and a few blocks' halves still do not fit and
    take the two-word or direct modes; 8 mm over 48 frames mixes one- and
    two-pass blocks.  Every shape stays bit-exact."""
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=48, grid=(270, 90, 200), y_start_mm=3.0, y_span_mm=span_mm)
    o = oracle_run(w)
    for cfg in [(128, 64, 16), (128, 64, 12), (128, 64, 11), (64, 32, 16), (128, 64, 8)]:
        g = run_with_tile(w, cfg)
        assert g["status"] == 0
        assert_pnn_bit_exact(g, o)


def test_pnn_tile_shapes_scalar_path():
    """Widths that are not a multiple of 8 take the per-byte loads."""
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn(seed=5, n=9, H=37, W=100, px=0.21, grid=(48, 40, 44), tilt_deg=15.0,
                       sweep_mm=5.0, y0_mm=3.0, band=(3, 30))
    o = oracle_run(w)
    for cfg in [(64, 16, 2), (256, 64, 8), (128, 5, 1)]:
        assert_pnn_bit_exact(run_with_tile(w, cfg), o)


def test_autotuner_pnn_keeps_a_valid_shape_and_stays_exact():
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=40, grid=(270, 80, 200), y_start_mm=3.0, y_span_mm=15.0)
    g = run_with_tile(w, None, tune=True)
    (tw, th, f), ms = g["tuned"]
    assert (tw, th, f) in PNN_SHAPES and ms > 0.0
    assert_pnn_bit_exact(g, oracle_run(w))
    vol = g["vol"]
    vol.set_tile(640, 480, None)  # back to the default
    assert vol.get_tile(640, 480) == (128, 64, 12)


def test_tile_config_errors():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=4, H=32, W=32, grid=(40, 40, 40))
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    for bad in [(96, 64, 8), (128, 0, 8), (128, 64, 17), (256, 64, 9), (128, 2000, 1),
                (128, 64, 0)]:
        with pytest.raises(usvol.UsvError) as e:
            vol.set_tile(32, 32, bad)
        assert e.value.code == usvol.ERR_RANGE
    for k in range(8):  # eight frame sizes fit, the ninth does not
        vol.set_tile(32 + k, 32, (64, 32, 4))
    with pytest.raises(usvol.UsvError) as e:
        vol.set_tile(100, 100, (64, 32, 4))
    assert e.value.code == usvol.ERR_RANGE
    tri = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear")
    for bad in [(128, 64, 4), (256, 129, 4), (256, 64, 9)]:
        with pytest.raises(usvol.UsvError):
            tri.set_tile(32, 32, bad)
    assert tri.get_tile(32, 32) == (256, 64, 4)
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    small = torch.empty(16, dtype=torch.int64, device="cuda")
    with pytest.raises(usvol.UsvError) as e:
        usvol.tune_insert(vol.handle, imgs.data_ptr(), 4, 32, 32, usvol.U8, poses.data_ptr(),
                          usvol.calibration_of(w), small.data_ptr(), 128)
    assert e.value.code == usvol.ERR_NOMEM


def test_trilinear_tile_shapes_within_tolerance():
    from paper_2412_00058_gb300 import synth
    w = synth.convex_fan(n=14, H=160, W=96, depth_mm=40.0, r0_mm=20.0, grid=(180, 60, 150),
                         spacing=0.4, band=(40, 70), sweep_mm=12.0, sway_mm=3.0, y_start_mm=6.0)
    o = oracle_run(w)
    for cfg in [(256, 16, 2), (256, 128, 8), (256, 33, 3), (256, 1, 1)]:
        g = run_with_tile(w, cfg)
        assert g["status"] == 0
        assert_trilinear_close(g, o)
    g = run_with_tile(w, None, tune=True)
    (tw, th, f), ms = g["tuned"]
    assert tw == 256 and th in (16, 32, 64, 128) and f in (2, 4, 8) and ms > 0.0
    assert_trilinear_close(g, o)
