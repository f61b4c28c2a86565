"""GPU parity of the trilinear splat variant (linear and convex probes, uint8
and float32 frames) against the FP64 oracle: |g - o| <= 1e-5 |o| + 1e-6
max|o| on S, W, filled values and the projection (voxels whose oracle
weight is below 2^-18 are left out of the S/W comparison: there the 2^-20
weight cut-off, taken in FP32 on the GPU and FP64 in the oracle, decides)."""
import numpy as np
import pytest

from helpers import assert_trilinear_close, build_library, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def convex_small(float_frames=False, n=24, seed=None):
    from paper_2412_00058_gb300 import synth
    kw = dict(n=n, H=160, W=96, depth_mm=40.0, r0_mm=20.0, grid=(180, 60, 150), spacing=0.4,
              band=(40, 70), sweep_mm=12.0, sway_mm=3.0, y_start_mm=6.0,
              float_frames=float_frames)
    if seed is not None:
        kw["seed"] = seed
    return synth.convex_fan(**kw)


def test_convex_fan_u8_matches_fp64_oracle():
    w = convex_small()
    g, o = gpu_run(w), oracle_run(w)
    assert g["status"] == 0 and o["skipped"] == 0
    assert_trilinear_close(g, o)


def test_convex_fan_f32_frames():
    w = convex_small(float_frames=True, n=10, seed=77)
    assert_trilinear_close(gpu_run(w), oracle_run(w))


def test_linear_probe_f32_pose_refinement_shape():
    from paper_2412_00058_gb300 import synth
    w = synth.pose_refine(n=40, H=96, W=80, grid=(80, 100, 70), spacing=0.3, band=(20, 50),
                          sweep_mm=20.0)
    g, o = gpu_run(w), oracle_run(w)
    assert_trilinear_close(g, o)


def test_trilinear_incremental_equals_batch_within_tolerance():
    w = convex_small(n=12, seed=5)
    a = gpu_run(w, splits=[5, 7])
    assert_trilinear_close(a, oracle_run(w))


def test_trilinear_bad_pose_skipped():
    from paper_2412_00058_gb300 import usvol
    w = convex_small(n=6, seed=9)
    w.poses[2, 1, 1] = np.inf
    g, o = gpu_run(w), oracle_run(w)
    assert o["skipped"] == 1 and g["status"] & usvol.STATUS_BAD_POSE
    assert_trilinear_close(g, o)


def _carry_run(w, carry):
    import torch
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear")
    vol.reset()
    imgs = torch.from_numpy(w.images).cuda()      # kept alive until the kernels have run
    poses = torch.from_numpy(w.poses).cuda()
    usvol.insert_trilinear_carry(vol.handle, imgs.data_ptr(), w.n, w.H, w.W,
                                 usvol.F32 if w.images.dtype == np.float32 else usvol.U8,
                                 poses.data_ptr(), usvol.calibration_of(w), carry)
    vol.fill()
    out, cnt = vol.project(*w.band)
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy()
    return dict(status=vol.status(), band=w.band, S=acc[..., 0].astype(np.float64),
                W=acc[..., 1].astype(np.float64), val=vol.read(usvol.READ_VALUES).cpu().numpy(),
                has=vol.read(usvol.READ_MASK).cpu().numpy(), proj=out.cpu().numpy(),
                pcnt=cnt.cpu().numpy().view(np.uint16))


def test_corner_carry_on_and_off_both_match_the_oracle():
    """The insertion kernel with the register carry of shared corner terms
    (what usv_insert_frames runs) and without it (what the pose-gradient
    path runs), on one convex and one linear batch: each against the FP64
    oracle, and the two against each other."""
    from helpers import close
    from paper_2412_00058_gb300 import synth
    lin = synth.pose_refine(n=24, H=96, W=80, grid=(80, 100, 70), spacing=0.3, band=(20, 50),
                            sweep_mm=12.0)
    for w in (convex_small(n=16, seed=21), lin):
        o = oracle_run(w)
        on, off = _carry_run(w, True), _carry_run(w, False)
        assert on["status"] == 0 and off["status"] == 0
        assert_trilinear_close(on, o)
        assert_trilinear_close(off, o)
        keep = o["W"] >= 2.0 ** -18
        for k in ("S", "W"):
            ok, worst = close(on[k], off[k], mask=keep)
            assert ok, f"carry on vs off, {k}: worst error / tolerance = {worst:.3g}"


def test_non_finite_and_huge_float_samples_are_not_inserted():
    """USV_F32 samples that are NaN, infinite or above 2^64 in magnitude are
    missing samples (no weight anywhere), on both sides: every other voxel
    matches the oracle, and no value or projection is NaN."""
    w = convex_small(float_frames=True, n=8, seed=31)
    rng = np.random.default_rng(4)
    imgs = w.images.copy()
    bad = [np.nan, np.inf, -np.inf, 3.0e38, -1.0e30, 2.0 ** 65]
    for k, v in enumerate(bad):
        f, i, j = rng.integers(0, w.n), rng.integers(10, w.H - 10), rng.integers(5, w.W - 5)
        imgs[f, i, j] = v
    imgs[3, 40:44, 30:34] = np.nan           # a block of them in one column walk
    g, o = gpu_run(w, images=imgs), oracle_run(w, images=imgs)
    assert g["status"] == 0
    for k in ("S", "W", "val", "proj"):
        assert np.all(np.isfinite(g[k])) and np.all(np.isfinite(o[k])), k
    assert_trilinear_close(g, o)
    # the dropped samples took their weight with them
    assert o["W"].sum() < oracle_run(w)["W"].sum()


def _fan_frames_reaching(w, y0, y1):
    """Frames whose y-extent (exact from the in-plane bounding box's 4
    corners: the map is affine) can reach voxel rows [y0, y1)."""
    import math
    half = math.radians(w.sector_deg) / 2
    R = w.r0 + (w.H - 1) * w.dr
    xs = (-R * math.sin(half), R * math.sin(half))
    zs = (w.r0 * math.cos(half) - w.r0, R - w.r0)
    keep = []
    for f in range(w.n):
        ys = [(w.poses[f] @ w.calib @ np.array([x, 0.0, z, 1.0]))[1] for x in xs for z in zs]
        qy0 = (min(ys) - w.origin[1]) / w.spacing[1]
        qy1 = (max(ys) - w.origin[1]) / w.spacing[1]
        if qy1 >= y0 - 2 and qy0 <= y1 + 1:
            keep.append(f)
    return keep


@pytest.mark.slow
def test_convex_fan_full_size_slabs_against_oracle():
    """Full-size convex sweep (3000 frames of 512x512 into 400x1700x400) in
    the launch configuration of the timed path.  The oracle recomputes four
    y-slabs of 12 voxel rows spread along the sweep -- where it starts and
    where it ends (only part of a frame group reaches them), and two inner
    ones -- each from the frames that can reach it, on a sub-grid of the slab
    plus two rows each side (insertion into a sub-grid is exact for every
    voxel inside it).  The GPU's S, W, filled values and depth-band
    projection must match on each slab's rows, with the trilinear
    tolerance."""
    import oracle
    from paper_2412_00058_gb300 import synth
    from helpers import close, effective_weight
    w = synth.convex_fan()
    g = gpu_run(w)
    assert g["status"] == 0
    nx, ny, nz = w.grid
    lo, hi = w.band
    compared = 0
    # the rows where the sweep starts and ends, and two between
    ys = [(w.poses[f] @ w.calib @ np.array([0.0, 0.0, 60.0, 1.0]))[1] for f in (0, w.n - 1)]
    first, last = (int((y - w.origin[1]) / w.spacing[1]) for y in ys)
    for y0 in (first - 6, 420, 800, last - 6):
        y1 = y0 + 12
        ya, yb = max(0, y0 - 2), min(ny, y1 + 2)
        keep = _fan_frames_reaching(w, ya, yb)
        assert 0 < len(keep) < w.n
        origin = (w.origin[0], w.origin[1] + ya * w.spacing[1], w.origin[2])
        S, Wt, sk = oracle.insert_trilinear((nx, yb - ya, nz), w.images[keep], w.poses[keep],
                                            w.calibration(), w.spacing, origin)
        assert sk == 0
        val, has = oracle.fill_trilinear(S, Wt)
        proj, pcnt = oracle.project_f64(val, has, lo, hi)
        rows = slice(y0 - ya, y1 - ya)
        gs = slice(y0, y1)
        m = Wt[:, rows, :] >= 2.0 ** -18
        for k, o in (("S", S), ("W", Wt)):
            ok, worst = close(g[k][:, gs, :], o[:, rows, :], mask=m)
            assert ok, f"slab {y0}: {k}: worst error / tolerance = {worst:.3g}"
        weff = effective_weight(Wt)[:, rows, :]
        both = (g["has"][:, gs, :] == 1) & (has[:, rows, :] == 1) & (weff >= 2.0 ** -18)
        ok, worst = close(g["val"][:, gs, :], val[:, rows, :], mask=both)
        assert ok, f"slab {y0}: values: worst error / tolerance = {worst:.3g}"
        decided = (weff >= 2.0 ** -18) | (weff == 0)
        assert np.array_equal(g["has"][:, gs, :][decided], has[:, rows, :][decided])
        weak = (has[:, rows, :] == 1) & (weff < 2.0 ** -18)
        cols = ~weak[lo:hi].any(axis=0)
        ok, worst = close(g["proj"][gs, :], proj[rows, :], mask=cols)
        assert ok, f"slab {y0}: projection: worst error / tolerance = {worst:.3g}"
        assert np.array_equal(g["pcnt"][gs, :][cols], pcnt[rows, :][cols])
        compared += int(m.sum())
    assert compared > 400_000
