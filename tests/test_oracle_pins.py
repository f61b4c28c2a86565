"""Pins of the CPU oracle against facts fixed by the method and by mathematics
(CPU only).  Each test names what it pins; none of them re-types the
oracle's own formula.

Method passages: Sec. II.C (PNN insertion: each pixel goes to its nearest
voxel, which keeps a sum and a hit count; its bin value is the mean; empty
bins are filled from neighbours), Alg. 1 steps 2-3/6 (pixels carried to the
world by calibration then the tracked pose T_T^W), Sec. III.B (VPI: a
coronal image from a fixed depth).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2412_00058_gb300 import synth

TWO32 = 1 << 32


def rigid(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


# ---------------------------------------------------------------- rounding

def test_round_half_away_ties_and_exact_values():
    assert oracle.round_half_away(2.5) == 3
    assert oracle.round_half_away(-2.5) == -3
    assert oracle.round_half_away(0.5) == 1
    assert oracle.round_half_away(-0.5) == -1
    assert oracle.round_half_away(1.4999999999999998) == 1
    assert oracle.round_half_away(2.0 ** 40 + 0.5) == 2 ** 40 + 1
    assert oracle.round_half_away(-(2.0 ** 40) - 0.5) == -(2 ** 40) - 1


# ---------------------------------------------------------------- A0: affine map

def test_affine_identity_translation_rotation_literals():
    s = (0.5, 0.5, 0.5)
    c, ok = oracle.frame_affine_q32(np.eye(4), np.eye(4), 0.5, 0.5, s, (0, 0, 0))
    assert ok
    assert list(c) == [TWO32, 0, 0, 0, 0, TWO32, 0, 0, 0]
    # translation by whole voxels -> C = (3, 5, 7) voxels
    c, ok = oracle.frame_affine_q32(rigid(np.eye(3), (1.5, 2.5, 3.5)), np.eye(4), 0.5, 0.5, s,
                                    (0, 0, 0))
    assert list(c[6:]) == [3 * TWO32, 5 * TWO32, 7 * TWO32]
    # 90 deg about z: image x axis -> world +y; image z axis unchanged
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    c, ok = oracle.frame_affine_q32(rigid(Rz, (0, 0, 0)), np.eye(4), 0.5, 0.5, s, (0, 0, 0))
    assert list(c[:3]) == [0, TWO32, 0] and list(c[3:6]) == [0, 0, TWO32]
    # calibration applied before the pose: K shifts the image by -1 mm in x,
    # then the pose rotates: world = Rz (x - 1, 0, z) -> C = Rz(-1,0,0)/0.5 = (0,-2,0)
    K = rigid(np.eye(3), (-1.0, 0.0, 0.0))
    c, ok = oracle.frame_affine_q32(rigid(Rz, (0, 0, 0)), K, 0.5, 0.5, s, (0, 0, 0))
    assert list(c[6:]) == [0, -2 * TWO32, 0]
    # origin and anisotropic spacing: C = (t - o)/s
    c, ok = oracle.frame_affine_q32(rigid(np.eye(3), (4.0, 4.0, 4.0)), np.eye(4), 1.0, 1.0,
                                    (0.5, 0.25, 2.0), (1.0, 2.0, 3.0))
    assert list(c[6:]) == [6 * TWO32, 8 * TWO32, TWO32 // 2]
    assert list(c[:3]) == [2 * TWO32, 0, 0] and list(c[3:6]) == [0, 0, TWO32 // 2]


def test_affine_invalid_frames():
    s = (0.5, 0.5, 0.5)
    bad = np.eye(4)
    bad[3, 0] = 1e-3                      # not an affine pose
    assert not oracle.frame_affine_q32(bad, np.eye(4), 0.5, 0.5, s, (0, 0, 0))[1]
    nanp = np.eye(4)
    nanp[0, 3] = np.nan
    assert not oracle.frame_affine_q32(nanp, np.eye(4), 0.5, 0.5, s, (0, 0, 0))[1]
    far = rigid(np.eye(3), (0.5 * 2 ** 29, 0, 0))   # |C| = 2^29 voxels: out of range
    assert not oracle.frame_affine_q32(far, np.eye(4), 0.5, 0.5, s, (0, 0, 0))[1]
    near = rigid(np.eye(3), (0.5 * (2 ** 29 - 1), 0, 0))
    assert oracle.frame_affine_q32(near, np.eye(4), 0.5, 0.5, s, (0, 0, 0))[1]


# ---------------------------------------------------------------- A1: PNN insertion

def _img(rng, H, W):
    return rng.integers(0, 256, size=(1, H, W), dtype=np.uint8)


def test_identity_pose_reproduces_image_in_one_slice():
    rng = np.random.default_rng(1)
    img = _img(rng, 12, 16)
    grid = (16, 8, 12)
    s, c, sk = oracle.insert_pnn(grid, img, rigid(np.eye(3), (0, 1.5, 0))[None], np.eye(4),
                                 0.5, 0.5, (0.5,) * 3, (0, 0, 0))
    assert sk == 0
    assert np.array_equal(s[:, 3, :], img[0].astype(np.uint64))
    assert np.all(c[:, 3, :] == 1)
    mask = np.ones(s.shape, bool)
    mask[:, 3, :] = False
    assert not s[mask].any() and not c[mask].any()


@pytest.mark.parametrize("shift", [(2, 3, -1), (-3, 0, 4), (0, 7, 0)])
def test_integer_translation_shifts_exactly(shift):
    rng = np.random.default_rng(2)
    img = _img(rng, 12, 16)
    grid = (16, 8, 12)
    dx, dy, dz = shift
    pose = rigid(np.eye(3), (0.5 * dx, 0.5 * dy, 0.5 * dz))
    s, c, _ = oracle.insert_pnn(grid, img, pose[None], np.eye(4), 0.5, 0.5, (0.5,) * 3, (0, 0, 0))
    exp_s = np.zeros_like(s)
    exp_c = np.zeros_like(c)
    for v in range(12):
        for u in range(16):
            x, y, z = u + dx, dy, v + dz
            if 0 <= x < 16 and 0 <= y < 8 and 0 <= z < 12:
                exp_s[z, y, x] += img[0, v, u]
                exp_c[z, y, x] += 1
    assert np.array_equal(s, exp_s) and np.array_equal(c, exp_c)


def test_half_voxel_ties_round_up():
    """Reading: nearest voxel with ties toward +inf.  A +1/2 voxel offset
    moves every pixel one voxel up, a -1/2 offset moves none."""
    rng = np.random.default_rng(3)
    img = _img(rng, 4, 6)
    grid = (8, 1, 4)
    up, _, _ = oracle.insert_pnn(grid, img, rigid(np.eye(3), (0.25, 0, 0))[None], np.eye(4),
                                 0.5, 0.5, (0.5,) * 3, (0, 0, 0))
    same, _, _ = oracle.insert_pnn(grid, img, rigid(np.eye(3), (-0.25, 0, 0))[None], np.eye(4),
                                   0.5, 0.5, (0.5,) * 3, (0, 0, 0))
    assert np.array_equal(up[:, 0, 1:7], img[0].astype(np.uint64))
    assert np.array_equal(same[:, 0, 0:6], img[0].astype(np.uint64))


def test_rotation_90_about_z_permutes_axes():
    rng = np.random.default_rng(4)
    img = _img(rng, 12, 16)
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    pose = rigid(Rz, (2.5, 0.5, 0))      # (u,0,v)*0.5 -> (2.5, 0.5 + 0.5u, 0.5v)
    s, c, _ = oracle.insert_pnn((8, 20, 12), img, pose[None], np.eye(4), 0.5, 0.5, (0.5,) * 3,
                                (0, 0, 0))
    for v in range(12):
        for u in range(16):
            assert s[v, u + 1, 5] == img[0, v, u] and c[v, u + 1, 5] == 1
    assert c.sum() == 12 * 16


def test_calibration_then_pose_order():
    """p = P K x: K first.  With K = 90 deg about y (image x -> world -z) and
    P a pure translation, rows of the image land along +x, columns along -z."""
    rng = np.random.default_rng(5)
    img = _img(rng, 3, 4)
    Ry = np.array([[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]])
    K = rigid(Ry, (0, 0, 0))             # (u,0,v)*0.5 -> (0.5v, 0, -0.5u)
    P = rigid(np.eye(3), (0.0, 0.0, 2.0))
    s, c, _ = oracle.insert_pnn((4, 1, 6), img, P[None], K, 0.5, 0.5, (0.5,) * 3, (0, 0, 0))
    for v in range(3):
        for u in range(4):
            assert s[4 - u, 0, v] == img[0, v, u]


def _compare_with_brute(w, limit_ambiguous=0):
    s, c, sk = oracle.insert_pnn(w.grid, w.images, w.poses, w.calib, w.sx, w.sy, w.spacing,
                                 w.origin)
    bs, bc, margin, inside = brute.pnn_brute(w.grid, w.images, w.poses, w.calib, w.sx, w.sy,
                                             w.spacing, w.origin)
    ambiguous = int((margin < 1e-7).sum())
    assert sk == 0
    assert ambiguous <= limit_ambiguous
    # total hits = number of in-volume pixels; total sum = their intensities
    assert int(c.sum(dtype=np.uint64)) == int(inside.sum())
    assert int(s.sum(dtype=np.uint64)) == int(w.images[inside].astype(np.uint64).sum())
    assert np.array_equal(s, bs) and np.array_equal(c, bc)
    return s, c


def test_random_tilted_sweep_matches_fp64_brute_force():
    w = synth.tiny_pnn(seed=11, n=6, H=40, W=36, grid=(40, 36, 44), band=(10, 20),
                       tilt_deg=12.0, sweep_mm=6.0, y0_mm=3.0)
    s, c = _compare_with_brute(w)
    assert 0 < c.sum() < w.n * w.H * w.W      # some pixels leave the volume


def test_fine_pixels_whole_spine_piece_matches_fp64_brute_force():
    w = synth.whole_spine(n=4, grid=(270, 30, 200), y_start_mm=2.0, y_span_mm=4.0)
    s, c = _compare_with_brute(w)
    # about 10 pixels of 0.083 x 0.094 mm per 0.3 mm voxel in a frame
    assert 5 < c[c > 0].mean() < 40


# ---------------------------------------------------------------- A2/A3: normalise + fill

def test_fill_closed_form_uniform_neighbourhood():
    s = np.full((3, 3, 3), 21, np.uint64)
    c = np.full((3, 3, 3), 2, np.uint32)
    s[1, 1, 1] = 0
    c[1, 1, 1] = 0
    val, has = oracle.fill_pnn(s, c)
    assert np.all(val == 11) and np.all(has == 1)     # 10.5 rounds half up


def test_fill_hand_built_pooled_means():
    s = np.zeros((3, 3, 3), np.uint64)
    c = np.zeros((3, 3, 3), np.uint32)
    s[0, 1, 1], c[0, 1, 1] = 100, 1      # A at (x=1, y=1, z=0)
    s[2, 1, 0], c[2, 1, 0] = 1, 3        # B at (x=0, y=1, z=2)
    val, has = oracle.fill_pnn(s, c)
    assert val[1, 1, 1] == 25 and has[1, 1, 1]       # (100 + 1) / (1 + 3) = 25.25
    assert val[0, 0, 0] == 100 and has[0, 0, 0]      # corner sees only A
    assert val[2, 2, 2] == 0 and not has[2, 2, 2]    # sees neither A nor B
    assert val[0, 1, 1] == 100 and val[2, 1, 0] == 0  # own means (1/3 -> 0)
    assert val[2, 2, 0] == 0 and has[2, 2, 0]        # sees only B: 1/3 -> 0
    assert val[1, 0, 2] == 100 and has[1, 0, 2]      # (x=2,y=0,z=1) sees only A
    assert val[1, 0, 1] == 25 and has[1, 0, 1]       # (x=1,y=0,z=1) sees A and B


def test_fill_rounding_ties_and_clamp():
    s = np.zeros((1, 1, 6), np.uint64)
    c = np.zeros((1, 1, 6), np.uint32)
    s[0, 0, :] = [5, 3, 1, 255 * 7, 0, 7]
    c[0, 0, :] = [2, 2, 2, 7, 1, 3]
    val, has = oracle.fill_pnn(s, c)
    assert list(val[0, 0]) == [3, 2, 1, 255, 0, 2] and has.all()


def test_fill_is_rounded_mean_without_holes_and_keeps_isolated_holes_empty():
    rng = np.random.default_rng(6)
    c = rng.integers(1, 40, size=(5, 6, 7)).astype(np.uint32)
    s = (c.astype(np.uint64) * rng.integers(0, 256, size=c.shape).astype(np.uint64))
    s = s - np.minimum(s, rng.integers(0, 3, size=c.shape).astype(np.uint64))
    val, has = oracle.fill_pnn(s, c)
    for idx in np.ndindex(c.shape):
        q = Fraction(int(s[idx]), int(c[idx])) + Fraction(1, 2)
        assert val[idx] == min(255, math.floor(q))
    e_s = np.zeros((5, 5, 5), np.uint64)
    e_c = np.zeros((5, 5, 5), np.uint32)
    e_s[0, 0, 0], e_c[0, 0, 0] = 9, 1
    val, has = oracle.fill_pnn(e_s, e_c)
    assert has.sum() == 8            # the voxel and its 7 in-grid neighbours
    assert not has[2, 2, 2]


# ---------------------------------------------------------------- A4: projection

def test_projection_constant_slice_and_literal():
    val = np.full((10, 4, 5), 7, np.uint8)
    has = np.ones_like(val)
    out, cnt = oracle.project_u8(val, has, 2, 9)
    assert np.all(out == 7.0) and np.all(cnt == 7)
    rng = np.random.default_rng(7)
    val = rng.integers(0, 256, size=(10, 4, 5)).astype(np.uint8)
    has = (rng.random((10, 4, 5)) < 0.6).astype(np.uint8)
    out, cnt = oracle.project_u8(val, has, 3, 4)
    assert np.array_equal(out, np.where(has[3], val[3], 0).astype(np.float32))
    assert np.array_equal(cnt, has[3].astype(np.uint16))
    out, cnt = oracle.project_u8(val, np.zeros_like(has), 0, 10)
    assert not out.any() and not cnt.any()
    v = np.zeros((4, 1, 1), np.uint8)
    h = np.zeros((4, 1, 1), np.uint8)
    v[:, 0, 0] = [10, 20, 31, 200]
    h[:, 0, 0] = [1, 1, 1, 0]
    out, cnt = oracle.project_u8(v, h, 0, 4)
    assert out[0, 0] == np.float32(61.0 / 3.0) and cnt[0, 0] == 3


def test_projection_is_linear_in_the_values_for_a_fixed_mask():
    """With the same has-data mask, the projection of V1 + V2 is the
    projection of V1 plus that of V2 (exactly, for values whose column sums
    divide evenly) and scaling V scales the projection."""
    rng = np.random.default_rng(23)
    has = (rng.random((12, 6, 7)) < 0.5).astype(np.uint8)
    _, cnt = oracle.project_u8(np.zeros_like(has), has, 2, 11)
    k = np.maximum(cnt.astype(np.int64), 1)
    # per column, values that are a multiple of the band count there: every
    # mean is an integer and exact in FP32
    base1 = rng.integers(0, 5, size=(12, 6, 7)) * k[None]
    base2 = rng.integers(0, 5, size=(12, 6, 7)) * k[None]
    v1 = np.minimum(base1, 120).astype(np.uint8)
    v2 = np.minimum(base2, 120).astype(np.uint8)
    p1, c1 = oracle.project_u8(v1, has, 2, 11)
    p2, c2 = oracle.project_u8(v2, has, 2, 11)
    p12, c12 = oracle.project_u8((v1 + v2).astype(np.uint8), has, 2, 11)
    assert np.array_equal(c1, c2) and np.array_equal(c1, c12)
    sums1 = (np.where(has[2:11], v1[2:11], 0).astype(np.int64)).sum(axis=0)
    sums2 = (np.where(has[2:11], v2[2:11], 0).astype(np.int64)).sum(axis=0)
    ok = (sums1 % k == 0) & (sums2 % k == 0)   # exact means on both sides
    assert ok.mean() > 0.5
    assert np.array_equal(p12[ok], (p1 + p2)[ok])
    p3, _ = oracle.project_u8((2 * v1).astype(np.uint8), has, 2, 11)
    assert np.array_equal(p3[ok], (2 * p1)[ok])


# ---------------------------------------------------------------- trilinear variant

def _single_frame(H, W, I, pose):
    imgs = np.zeros((1, H, W), np.float32)
    imgs[0] = I
    return imgs, pose[None]


def test_trilinear_voxel_centre_sample_hits_one_voxel():
    imgs, poses = _single_frame(1, 1, 5.0, rigid(np.eye(3), (1.5, 2.0, 2.5)))
    cal = dict(image_to_probe=np.eye(4), sx=0.5, sy=0.5, geom="linear")
    S, Wt, _ = oracle.insert_trilinear((6, 6, 6), imgs, poses, cal, (0.5,) * 3, (0, 0, 0))
    assert S[5, 4, 3] == 5.0 and Wt[5, 4, 3] == 1.0
    assert np.count_nonzero(Wt) == 1


def test_trilinear_convex_sample_position_closed_form():
    """A single unit sample's splat has its weighted centroid at the sample
    (trilinear weights reproduce linear functions).  Convex geometry, beam j
    at theta = -30 + j*10 deg (7 beams over 60 deg), r = r0 + i*dr."""
    H, W = 4, 7
    imgs = np.zeros((1, H, W), np.float32)
    imgs[0, 2, 0] = 1.0                          # i = 2, j = 0
    centre = np.array([20.0, 20.0, 10.0])
    cal = dict(image_to_probe=np.eye(4), geom="convex", r0=10.0, dr=1.0, sector_deg=60.0)
    S, Wt, _ = oracle.insert_trilinear((40, 40, 40), imgs, rigid(np.eye(3), centre)[None], cal,
                                       (1.0,) * 3, (0, 0, 0))
    zz, yy, xx = np.nonzero(S)
    w = S[zz, yy, xx]
    cen = np.array([np.dot(w, xx), np.dot(w, yy), np.dot(w, zz)]) / w.sum()
    expect = centre + np.array([-6.0, 0.0, 6.0 * math.sqrt(3.0) - 10.0])   # r = 12, -30 deg
    assert np.allclose(cen, expect, atol=1e-9)
    assert abs(w.sum() - 1.0) < 8 * 2.0 ** -20


def _voxel_positions(w):
    """FP64 sample positions in voxel units, computed from the geometry."""
    n, H, W = w.images.shape
    ii, jj = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    if w.geom == "convex":
        half = math.radians(w.sector_deg) / 2
        th = -half + jj * (2 * half / (W - 1))
        r = w.r0 + ii * w.dr
        x, z = r * np.sin(th), r * np.cos(th) - w.r0
    else:
        x, z = jj * w.sx, ii * w.sy
    pts = np.stack([x, np.zeros_like(x), z, np.ones_like(x)], -1)
    M = np.einsum("fij,jk->fik", w.poses, w.calib)
    p = np.einsum("fij,hwj->fhwi", M, pts)[..., :3]
    return (p - np.asarray(w.origin)) / np.asarray(w.spacing)


@pytest.mark.parametrize("geom", ["linear", "convex"])
def test_trilinear_splat_is_adjoint_of_trilinear_interpolation(geom):
    """<splat(I), V> = sum_s I_s * interp(V, q_s) for any V, with scipy's
    order-1 map_coordinates as the interpolation (out-of-grid corners read 0);
    weights below 2^-20 dropped by the splat bound the difference."""
    from scipy.ndimage import map_coordinates
    if geom == "convex":
        w = synth.convex_fan(n=3, H=24, W=20, depth_mm=8.0, r0_mm=6.0, grid=(48, 40, 36),
                             spacing=0.4, sweep_mm=2.0, sway_mm=0.0, y_start_mm=7.0,
                             float_frames=True)
    else:
        w = synth.pose_refine(n=3, H=20, W=24, px=0.2, grid=(40, 30, 30), spacing=0.3,
                              sweep_mm=2.0)
        w.poses[:, 1, 3] = np.array([3.0, 3.7, 4.4])
        w.poses[:, 0, 3] = 6.0
    S, Wt, sk = oracle.insert_trilinear(w.grid, w.images, w.poses, w.calibration(), w.spacing,
                                        w.origin)
    assert sk == 0
    q = _voxel_positions(w).reshape(-1, 3)
    rng = np.random.default_rng(8)
    V = rng.normal(size=S.shape)
    coords = np.stack([q[:, 2], q[:, 1], q[:, 0]])       # V is [z, y, x]
    interp = map_coordinates(V, coords, order=1, mode="grid-constant", cval=0.0)
    I = w.images.reshape(-1).astype(np.float64)
    bound = 8 * 2.0 ** -20 * np.abs(V).max() * (np.abs(I).sum() + len(I)) + 1e-9
    assert abs(np.vdot(S, V) - np.dot(I, interp)) <= bound
    assert abs(np.vdot(Wt, V) - interp.sum()) <= bound
    assert Wt.sum() > 0


def test_trilinear_partition_of_unity_for_interior_frames():
    w = synth.pose_refine(n=4, H=16, W=16, px=0.2, grid=(40, 40, 40), spacing=0.3, sweep_mm=1.5)
    w.poses[:, 0, 3] = 5.0
    w.poses[:, 1, 3] = 4.0 + np.arange(4) * 0.37
    S, Wt, _ = oracle.insert_trilinear(w.grid, w.images, w.poses, w.calibration(), w.spacing,
                                       w.origin)
    nsamp = w.n * w.H * w.W
    assert abs(Wt.sum() - nsamp) <= nsamp * 8 * 2.0 ** -20
    assert abs(S.sum() - w.images.astype(np.float64).sum()) <= 255 * nsamp * 8 * 2.0 ** -20


def test_trilinear_fill_and_projection_closed_forms():
    S = np.zeros((3, 3, 3))
    Wt = np.zeros((3, 3, 3))
    S[0, 1, 1], Wt[0, 1, 1] = 30.0, 0.5
    S[2, 1, 0], Wt[2, 1, 0] = 3.0, 1.5
    val, has = oracle.fill_trilinear(S, Wt)
    assert val[0, 1, 1] == 60.0 and val[2, 1, 0] == 2.0
    assert val[1, 1, 1] == 33.0 / 2.0            # pooled: (30 + 3) / (0.5 + 1.5)
    assert not has[2, 2, 2]
    out, cnt = oracle.project_f64(val, has, 0, 3)
    assert cnt[1, 1] == 3 and math.isclose(out[1, 1], (60.0 + 16.5 + val[2, 1, 1]) / 3)


def test_multi_core_oracle_gives_the_single_thread_bits():
    """The OpenMP forms (frames split over host threads with atomic integer
    adds; fill and projection split by plane / row) reproduce the plain
    single-thread loops bit for bit."""
    import oracle
    from paper_2412_00058_gb300 import synth
    w = synth.whole_spine(n=60, grid=(270, 80, 200), y_start_mm=3.0, y_span_mm=20.0)
    cut = np.arange(w.n, dtype=np.int32) % 7 * 11
    ref = []
    try:
        for t in (1, 4):
            got = oracle.set_threads(t)
            assert got == t or got == 1
            s, c, sk = oracle.insert_pnn(w.grid, w.images, w.poses, w.calib, w.sx, w.sy,
                                         w.spacing, w.origin, first_rows=cut)
            v, h = oracle.fill_pnn(s, c)
            p, pc = oracle.project_u8(v, h, *w.band)
            ref.append((s, c, sk, v, h, p, pc))
    finally:
        oracle.set_threads(1)
    for a, b in zip(*ref):
        assert np.array_equal(a, b)
    assert ref[0][1].sum() > 0
