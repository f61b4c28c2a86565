"""Saving and resuming a scan: the accumulator file format on the CPU, and on
the GPU a scan saved half-way, loaded into a new volume and finished, which
must equal the oracle of the whole scan bit for bit (PNN accumulators are
integers), plus the end-of-scan slices along the spine axis."""
import os

import numpy as np
import pytest

from helpers import assert_pnn_bit_exact, gpu_run, oracle_run


def test_volume_file_round_trip_and_rejections(tmp_path):
    from paper_2412_00058_gb300 import usvol
    rng = np.random.default_rng(7)
    acc = rng.integers(0, 2 ** 40, size=(3, 4, 5), dtype=np.int64)
    meta = dict(grid=[5, 4, 3], spacing=[0.3, 0.4, 0.5], origin=[1.0, -2.0, 0.25], mode="pnn")
    p = tmp_path / "v.usv"
    usvol.write_volume_file(p, meta, acc)
    head, back = usvol.read_volume_file(p)
    assert np.array_equal(back, acc) and back.dtype == np.int64
    assert head["grid"] == [5, 4, 3] and head["spacing"] == [0.3, 0.4, 0.5]
    assert head["origin"] == [1.0, -2.0, 0.25] and head["mode"] == "pnn"
    tri = rng.standard_normal((3, 4, 5, 2)).astype(np.float32)
    usvol.write_volume_file(p, dict(meta, mode="trilinear"), tri)
    head, back = usvol.read_volume_file(p)
    assert np.array_equal(back, tri) and head["mode"] == "trilinear"
    # a foreign file, a truncated one, and a shape that does not match the grid
    (tmp_path / "x").write_bytes(b"not a volume at all")
    with pytest.raises(ValueError):
        usvol.read_volume_file(tmp_path / "x")
    data = p.read_bytes()
    (tmp_path / "t").write_bytes(data[:-4])
    with pytest.raises(ValueError):
        usvol.read_volume_file(tmp_path / "t")
    usvol.write_volume_file(p, dict(meta, grid=[5, 4, 4]), acc)
    with pytest.raises(ValueError):
        usvol.read_volume_file(p)


@pytest.mark.gpu
def test_scan_saved_half_way_resumes_bit_exactly(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.whole_spine(n=40, grid=(270, 80, 200), y_start_mm=5.0, y_span_mm=14.0)
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    cal = usvol.calibration_of(w)
    first = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    first.reset()
    first.insert(imgs[:17], poses[:17], cal)
    path = tmp_path / "half.usv"
    first.save(path)
    del first
    vol = usvol.Volume.load(path, spare=True)
    assert vol.grid == w.grid and vol.spacing == tuple(w.spacing) and vol.origin == w.origin
    vol.insert(imgs[17:], poses[17:], cal)
    vol.fill()
    out, cnt = vol.project(*w.band)
    assert vol.status() == 0
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    g = dict(sum=acc & np.uint64(0xFFFFFFFF), cnt=(acc >> np.uint64(32)).astype(np.uint32),
             val=vol.read(usvol.READ_VALUES).cpu().numpy(),
             has=vol.read(usvol.READ_MASK).cpu().numpy(), proj=out.cpu().numpy(),
             pcnt=cnt.cpu().numpy().view(np.uint16))
    o = oracle_run(w)
    assert_pnn_bit_exact(g, o)
    # the end-of-scan slices along y: depth down, lateral across
    names = vol.save_slices(tmp_path / "slices")
    assert len(names) == w.grid[1]
    for y in (0, 37, w.grid[1] - 1):
        raw = open(names[y], "rb").read()
        head = b"P5\n%d %d\n255\n" % (w.grid[0], w.grid[2])
        assert raw.startswith(head)
        img = np.frombuffer(raw[len(head):], np.uint8).reshape(w.grid[2], w.grid[0])
        assert np.array_equal(img, o["val"][:, y, :])


@pytest.mark.gpu
def test_trilinear_volume_saves_and_loads_exactly(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.convex_fan(n=12, H=160, W=96, depth_mm=40.0, r0_mm=20.0, grid=(180, 60, 150),
                         spacing=0.4, band=(40, 70), sweep_mm=12.0, sway_mm=3.0, y_start_mm=6.0)
    g = gpu_run(w)
    path = tmp_path / "tri.usv"
    g["vol"].save(path)
    vol = usvol.Volume.load(path)
    assert vol.mode == usvol.TRILINEAR
    a = g["vol"].read(usvol.READ_ACCUM).cpu().numpy()
    b = vol.read(usvol.READ_ACCUM).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
