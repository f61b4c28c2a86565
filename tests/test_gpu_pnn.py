"""GPU parity of the nearest-neighbour path (insert, fill, project) against the
CPU oracle, through the C ABI.  Bit-exact: the path is integer end to end
except the final FP32 division of the projection, which both sides take as
one correctly rounded division of exact values."""
import numpy as np
import pytest

from helpers import assert_pnn_bit_exact, build_library, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def test_tiny_pnn_config_bit_exact():
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn()
    g, o = gpu_run(w), oracle_run(w)
    assert g["status"] == 0 and o["skipped"] == 0
    assert_pnn_bit_exact(g, o)
    assert o["cnt"].sum() > 500_000


def test_whole_spine_piece_bit_exact_many_tiles_ragged_tail():
    """480x640 frames: 128-column tiles leave a 96-column tail, 64-row tiles;
    48 frames span several frame groups with a ragged last group."""
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=47, grid=(270, 90, 200), y_start_mm=3.0, y_span_mm=20.0)
    g, o = gpu_run(w), oracle_run(w)
    assert g["status"] == 0
    assert_pnn_bit_exact(g, o)


@pytest.mark.parametrize("H,W", [(37, 100), (64, 33), (5, 7)])
def test_scalar_load_path_for_ragged_widths(H, W):
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn(seed=5, n=9, H=H, W=W, px=0.21, grid=(48, 40, 44), tilt_deg=15.0,
                       sweep_mm=5.0, y0_mm=3.0, band=(3, 30))
    assert_pnn_bit_exact(gpu_run(w), oracle_run(w))


def test_misaligned_frame_pointer_takes_scalar_path():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(seed=6, n=5, H=32, W=32, px=0.25, grid=(40, 40, 40), sweep_mm=4.0,
                       y0_mm=2.0, band=(0, 40))
    buf = torch.empty(w.images.size + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = torch.from_numpy(w.images.reshape(-1)).cuda()
    imgs = buf[1:].view(w.images.shape)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    vol.reset()
    vol.insert(imgs, torch.from_numpy(w.poses).cuda(), usvol.calibration_of(w))
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    o = oracle_run(w)
    assert np.array_equal(acc & np.uint64(0xFFFFFFFF), o["sum"])
    assert np.array_equal(acc >> np.uint64(32), o["cnt"].astype(np.uint64))


def test_incremental_inserts_equal_one_batch():
    """The paper's incremental method: inserting frames in uneven batches on
    top of the existing volume gives the same volume as one call."""
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=30, grid=(270, 60, 200), y_start_mm=5.0, y_span_mm=10.0)
    a = gpu_run(w, splits=[1, 7, 3, 19])
    b = gpu_run(w)
    for k in ("sum", "cnt", "val", "has", "proj"):
        assert np.array_equal(a[k], b[k])
    assert_pnn_bit_exact(a, oracle_run(w))


def test_more_frames_than_one_setup_chunk():
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn(seed=7, n=4100, H=16, W=16, px=0.3, grid=(24, 64, 24), tilt_deg=5.0,
                       sweep_mm=16.0, y0_mm=1.0, band=(2, 20))
    assert_pnn_bit_exact(gpu_run(w), oracle_run(w))


def test_frames_outside_volume_and_empty_batch():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(seed=8, n=4, H=32, W=32, grid=(32, 32, 32), band=(0, 32))
    w.poses[:, 1, 3] += 500.0                     # far along y: nothing lands
    g = gpu_run(w)
    assert g["cnt"].sum() == 0 and g["has"].sum() == 0 and not g["proj"].any()
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    vol.reset()
    e = torch.empty((0, 32, 32), dtype=torch.uint8, device="cuda")
    p = torch.empty((0, 4, 4), dtype=torch.float64, device="cuda")
    vol.insert(e, p, usvol.calibration_of(w))
    assert vol.status() == 0


def test_bad_poses_are_skipped_and_reported():
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(seed=9, n=12, H=48, W=48, grid=(64, 64, 64), band=(10, 40))
    w.poses[3, 0, 3] = np.nan
    w.poses[5, 3, 0] = 1e-3                       # not affine
    w.poses[7, 2, 3] = 1e12                       # out of range
    g, o = gpu_run(w), oracle_run(w)
    assert o["skipped"] == 3
    assert g["status"] & usvol.STATUS_BAD_POSE
    assert_pnn_bit_exact(g, o)


def test_steep_and_coarse_frames_use_direct_atomics():
    """Pixels larger than voxels and 60-degree tilts make tile boxes exceed
    shared memory: those tiles send runs straight to HBM atomics."""
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn(seed=10, n=6, H=128, W=128, px=0.9, grid=(100, 100, 100),
                       tilt_deg=60.0, sweep_mm=10.0, y0_mm=12.0, band=(20, 60))
    assert_pnn_bit_exact(gpu_run(w), oracle_run(w))


@pytest.mark.parametrize("tile", [(64, 32, 8), (128, 64, 8), (256, 128, 8)])
def test_frames_larger_than_the_grid(tile):
    """Every tile is clipped by a grid smaller than the frames (and shifted
    off-centre, so boxes start before the grid on some axes): tiles whose
    whole box fits keep it and drop the out-of-grid entries at the flush,
    the larger ones clip their box and check their segments; either way the
    volume equals the oracle's."""
    from paper_2412_00058_gb300 import synth
    w = synth.tiny_pnn(seed=12, n=16, H=256, W=256, px=0.3, grid=(40, 30, 50),
                       tilt_deg=20.0, sweep_mm=6.0, y0_mm=2.0, band=(5, 40))
    w.poses[:, 0, 3] += 2.0                       # the grid sits off the frames' centre
    g = gpu_run_tile(w, tile)
    assert g["status"] == 0
    o = oracle_run(w)
    assert o["cnt"].sum() > 5000                  # the grid does receive pixels
    assert_pnn_bit_exact(g, o)


def gpu_run_tile(w, tile):
    import torch
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume(w.grid, w.spacing, w.origin, w.mode)
    vol.set_tile(w.H, w.W, tile)
    vol.reset()
    vol.insert(torch.from_numpy(w.images).cuda(), torch.from_numpy(w.poses).cuda(),
               usvol.calibration_of(w))
    vol.fill()
    out, cnt = vol.project(*w.band)
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    return dict(status=vol.status(), sum=acc & np.uint64(0xFFFFFFFF),
                cnt=(acc >> np.uint64(32)).astype(np.uint32),
                val=vol.read(usvol.READ_VALUES).cpu().numpy(),
                has=vol.read(usvol.READ_MASK).cpu().numpy(), proj=out.cpu().numpy(),
                pcnt=cnt.cpu().numpy().view(np.uint16))


def test_fill_and_projection_on_hand_built_accumulators():
    """Sparse random accumulators (holes everywhere, grid borders, nx not a
    multiple of 32, ny not of 8) written through usv_volume_write_accum."""
    import torch
    import oracle
    from paper_2412_00058_gb300 import usvol
    rng = np.random.default_rng(12)
    for grid in [(45, 13, 7), (32, 8, 1), (1, 1, 5), (70, 3, 40)]:
        nx, ny, nz = grid
        c = np.where(rng.random((nz, ny, nx)) < 0.3, rng.integers(1, 50, (nz, ny, nx)), 0)
        s = (c * rng.integers(0, 256, (nz, ny, nx))).astype(np.uint64)
        c = c.astype(np.uint32)
        packed = (c.astype(np.uint64) << np.uint64(32)) | s
        vol = usvol.Volume(grid, (0.5, 0.5, 0.5), (0, 0, 0), "pnn")
        src = torch.from_numpy(packed.view(np.int64)).cuda()
        usvol.volume_write_accum(vol.handle, src.data_ptr())
        vol.fill()
        for lo, hi in [(0, nz), (nz - 1, nz), (0, 1)]:
            out, cnt = vol.project(lo, hi)
            ov, oh = oracle.fill_pnn(s, c)
            op, oc = oracle.project_u8(ov, oh, lo, hi)
            assert np.array_equal(out.cpu().numpy(), op)
            assert np.array_equal(cnt.cpu().numpy().view(np.uint16), oc)
        assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), ov)
        assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), oh)


def test_projection_word_kernel_grids_and_pointer_alignments():
    """Whole-plane projections take 4 columns per thread where the plane
    allows 32-bit words; grids whose 4-column groups wrap rows (nx not a
    multiple of 4), cross 32-column mask words, or would span three mask
    words (nx = 1 or 2 mod 32, taken by the one-column kernel), and outputs
    at 16-byte, 4-byte and 2-byte alignments, with and without counts, all
    equal the oracle."""
    import torch
    import oracle
    from paper_2412_00058_gb300 import usvol
    rng = np.random.default_rng(77)
    for grid in [(270, 12, 20), (45, 4, 9), (63, 4, 9), (31, 4, 5), (33, 4, 6), (66, 2, 6),
                 (36, 5, 12), (45, 3, 4)]:
        nx, ny, nz = grid
        c = np.where(rng.random((nz, ny, nx)) < 0.3, rng.integers(1, 50, (nz, ny, nx)), 0)
        s = (c * rng.integers(0, 256, (nz, ny, nx))).astype(np.uint64)
        c = c.astype(np.uint32)
        packed = (c.astype(np.uint64) << np.uint64(32)) | s
        vol = usvol.Volume(grid, (0.5, 0.5, 0.5), (0, 0, 0), "pnn")
        src = torch.from_numpy(packed.view(np.int64)).cuda()
        usvol.volume_write_accum(vol.handle, src.data_ptr())
        vol.fill()
        ov, oh = oracle.fill_pnn(s, c)
        n = nx * ny
        for lo, hi in [(0, nz), (1, nz), (nz - 1, nz)]:
            op, oc = oracle.project_u8(ov, oh, lo, hi)
            for off_out, off_cnt, with_cnt in [(0, 0, True), (1, 1, True), (4, 4, True),
                                               (0, 0, False), (1, 0, False)]:
                out = torch.full((n + 8,), -1.0, dtype=torch.float32, device="cuda")
                cnt = torch.full((n + 8,), 7, dtype=torch.int16, device="cuda")
                usvol.project_depth_band(vol.handle, lo, hi, out.data_ptr() + 4 * off_out,
                                         cnt.data_ptr() + 2 * off_cnt if with_cnt else None)
                torch.cuda.synchronize()
                o = out.cpu().numpy()
                assert np.array_equal(o[off_out:off_out + n].reshape(ny, nx), op), (grid, lo, off_out)
                assert (o[:off_out] == -1.0).all() and (o[off_out + n:] == -1.0).all()
                k = cnt.cpu().numpy().view(np.uint16)
                if with_cnt:
                    assert np.array_equal(k[off_cnt:off_cnt + n].reshape(ny, nx), oc)
                    assert (k[:off_cnt] == 7).all() and (k[off_cnt + n:] == 7).all()
                else:
                    assert (k == 7).all()


def test_fill_large_accumulators_both_plane_loaders():
    """Counts at and above 2^24 (the fill's 64-bit path and the saturation
    flag) next to ordinary planes, on an even nx (planes arrive by tensor
    copies) and an odd nx (per-entry asynchronous copies): both equal the
    oracle bit for bit."""
    import torch
    import oracle
    from paper_2412_00058_gb300 import usvol
    rng = np.random.default_rng(31)
    for grid in [(64, 37, 9), (63, 37, 9), (96, 70, 5)]:
        nx, ny, nz = grid
        c = np.where(rng.random((nz, ny, nx)) < 0.4, rng.integers(1, 40, (nz, ny, nx)), 0)
        big = rng.random((nz, ny, nx)) < 0.02
        big[nz // 2] = False            # a plane far from any large count
        big[:, :, : nx // 3] = False    # columns whose neighbourhood stays small
        c = np.where(big, rng.integers(1 << 23, 1 << 26, (nz, ny, nx)), c)
        s = (c * rng.integers(0, 64, (nz, ny, nx))).astype(np.uint64)
        assert int(s.max()) < 1 << 32
        c = c.astype(np.uint32)
        packed = (c.astype(np.uint64) << np.uint64(32)) | s
        vol = usvol.Volume(grid, (0.5, 0.5, 0.5), (0, 0, 0), "pnn")
        src = torch.from_numpy(packed.view(np.int64)).cuda()
        usvol.volume_write_accum(vol.handle, src.data_ptr())
        vol.fill()
        ov, oh = oracle.fill_pnn(s, c)
        assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), ov)
        assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), oh)
        saturated = bool((c >= (1 << 24)).any())
        assert bool(vol.status() & usvol.STATUS_SATURATED) == saturated
        assert not vol.status() & usvol.STATUS_TIMEOUT


def _random_accumulators(rng, grid):
    nx, ny, nz = grid
    c = np.where(rng.random((nz, ny, nx)) < 0.35, rng.integers(1, 60, (nz, ny, nx)), 0)
    s = (c * rng.integers(0, 256, (nz, ny, nx))).astype(np.uint64)
    c = c.astype(np.uint32)
    return s, c, (c.astype(np.uint64) << np.uint64(32)) | s


@pytest.mark.parametrize("grid,spare", [((64, 37, 40), True),    # fused, tensor copies
                                        ((63, 37, 40), True),    # fused, odd nx
                                        ((64, 37, 40), False)])  # fill, then reset
def test_fill_and_clear(grid, spare):
    """fill_and_clear gives the fill's values and mask, leaves the
    accumulators zero (every voxel, across several z slabs), and the next
    sweep on the same volume equals a fresh volume."""
    import torch
    import oracle
    from paper_2412_00058_gb300 import synth, usvol
    rng = np.random.default_rng(5)
    vol = usvol.Volume(grid, (0.3, 0.3, 0.3), (0, 0, 0), "pnn", spare=spare)
    for sweep in range(2):
        s, c, packed = _random_accumulators(rng, grid)
        src = torch.from_numpy(packed.view(np.int64)).cuda()
        usvol.volume_write_accum(vol.handle, src.data_ptr())
        vol.fill_and_clear()
        ov, oh = oracle.fill_pnn(s, c)
        assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), ov)
        assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), oh)
        assert not vol.read(usvol.READ_ACCUM).cpu().numpy().any()
    w = synth.tiny_pnn(n=12, H=48, W=40, grid=grid, band=(10, 20), sweep_mm=2.0, y0_mm=4.0)
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    cal = usvol.calibration_of(w)
    vol.insert(imgs, poses, cal)
    vol.fill_and_clear()
    fresh = usvol.Volume(grid, (0.3, 0.3, 0.3), (0, 0, 0), "pnn")
    fresh.reset()
    fresh.insert(imgs, poses, cal)
    fresh.fill()
    assert fresh.read(usvol.READ_ACCUM).cpu().numpy().any()
    for what in (usvol.READ_VALUES, usvol.READ_MASK):
        assert np.array_equal(vol.read(what).cpu().numpy(), fresh.read(what).cpu().numpy())
    assert not vol.read(usvol.READ_ACCUM).cpu().numpy().any()
    assert vol.status() == 0


def test_fill_and_clear_trilinear_is_fill_then_reset():
    import torch
    from paper_2412_00058_gb300 import usvol
    grid = (40, 20, 18)
    rng = np.random.default_rng(8)
    sw = np.zeros((18, 20, 40, 2), np.float32)
    m = rng.random((18, 20, 40)) < 0.3
    sw[m, 1] = rng.random(m.sum()).astype(np.float32) + 0.1
    sw[m, 0] = sw[m, 1] * rng.integers(0, 256, m.sum())
    a = usvol.Volume(grid, (0.4,) * 3, (0, 0, 0), "trilinear", spare=True)
    b = usvol.Volume(grid, (0.4,) * 3, (0, 0, 0), "trilinear")
    src = torch.from_numpy(sw.view(np.int64)).cuda()
    for v in (a, b):
        usvol.volume_write_accum(v.handle, src.data_ptr())
    a.fill_and_clear()
    b.fill()
    for what in (usvol.READ_VALUES, usvol.READ_MASK):
        assert np.array_equal(a.read(what).cpu().numpy(), b.read(what).cpu().numpy())
    assert not a.read(usvol.READ_ACCUM).cpu().numpy().any()


def test_argument_errors_with_a_live_volume():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=2, H=16, W=16)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    L = usvol.lib()
    cal = usvol.calibration_of(w)
    sp = usvol._stream_ptr(None)

    def ins(im=imgs.data_ptr(), n=2, H=16, W=16, dt=0, ps=poses.data_ptr(), c=cal):
        import ctypes
        return L.usv_insert_frames_dev(vol.handle, im, n, H, W, dt, ps, ctypes.byref(c), sp)

    assert ins(n=-1) == usvol.ERR_ARG
    assert ins(H=0) == usvol.ERR_ARG
    assert ins(W=40000) == usvol.ERR_RANGE
    assert ins(dt=1) == usvol.ERR_UNSUPPORTED           # PNN takes uint8 frames
    assert ins(ps=poses.data_ptr() + 4) == usvol.ERR_ARG
    bad = usvol.calibration_of(w)
    bad.image_to_probe[12] = 1.0
    assert ins(c=bad) == usvol.ERR_ARG
    bad = usvol.calibration_of(w)
    bad.sx_mm = 0.0
    assert ins(c=bad) == usvol.ERR_ARG
    convex = usvol.make_calibration(np.eye(4), "convex", r0=40, dr=0.2, sector_deg=60)
    assert ins(c=convex) == usvol.ERR_UNSUPPORTED       # PNN is linear-probe only
    out = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    assert L.usv_project_depth_band(vol.handle, 5, 5, out.data_ptr(), None, sp) == usvol.ERR_RANGE
    assert L.usv_project_depth_band(vol.handle, 0, 129, out.data_ptr(), None, sp) == usvol.ERR_RANGE
    assert L.usv_fill_holes(vol.handle, 2, sp) == usvol.ERR_UNSUPPORTED
    assert vol.status() == 0


def test_deterministic_across_runs():
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=20, grid=(270, 50, 200), y_start_mm=8.0, y_span_mm=8.0)
    a, b = gpu_run(w), gpu_run(w)
    for k in ("sum", "cnt", "val", "has", "proj", "pcnt"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.slow
def test_whole_spine_full_size_bit_exact():
    """The full whole-spine sweep (3600 frames of 480x640 into 270x1840x200),
    in the single launch the benchmark times, against the full oracle."""
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine()
    g = gpu_run(w)
    o = oracle_run(w)
    assert g["status"] == 0 and o["skipped"] == 0
    assert_pnn_bit_exact(g, o)


def test_host_poses_through_the_staging_ring_equal_device_poses_and_the_oracle():
    """usv_insert_frames takes host poses (the tracker's output) and stages
    them through the volume's pinned ring: calls of 4500 (two launches),
    300, 1 and 199 frames, several times over so that the 2 MB ring wraps,
    give exactly the volume of device-pose calls and of the oracle."""
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=5000, H=16, W=32, sweep_mm=20.0)
    imgs = torch.from_numpy(w.images).cuda()
    cal = usvol.calibration_of(w)
    a = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    b = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    a.reset()
    b.reset()
    d_poses = torch.from_numpy(w.poses).cuda()
    reps = 4                       # 4 x 640 KB of poses: the 2 MB ring wraps
    for _ in range(reps):
        f = 0
        for k in (4500, 300, 1, 199):
            a.insert(imgs[f:f + k], w.poses[f:f + k], cal)              # host poses
            b.insert(imgs[f:f + k], d_poses[f:f + k], cal)              # device poses
            f += k
    assert a.status() == 0 and b.status() == 0
    acc_a = a.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    assert np.array_equal(acc_a, b.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64))
    import oracle
    s, c, _ = oracle.insert_pnn(w.grid, w.images, w.poses, w.calib, w.sx, w.sy, w.spacing,
                                w.origin)
    assert np.array_equal(acc_a & np.uint64(0xFFFFFFFF), s * np.uint64(reps))
    assert np.array_equal(acc_a >> np.uint64(32), c.astype(np.uint64) * np.uint64(reps))
