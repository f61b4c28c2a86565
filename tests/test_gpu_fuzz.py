"""Seeded random geometries against the oracle, bit for bit: frame sizes
(odd widths included), pixel sizes from much finer to coarser than the
voxels, anisotropic voxels, origin offsets, tilts up to 60 degrees, frames
partly outside the grid, and random tile shapes -- so the packed, split and
direct accumulation modes, clipped and unclipped tiles and the per-byte
loads all meet the oracle."""
import dataclasses

import numpy as np
import pytest

from helpers import assert_pnn_bit_exact, build_library, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def random_case(k: int):
    from paper_2412_00058_gb300 import synth
    rng = np.random.default_rng(1000 + k)
    H, W = int(rng.integers(3, 200)), int(rng.integers(3, 260))
    n = int(rng.integers(1, 40))
    px = float(np.exp(rng.uniform(np.log(0.05), np.log(0.7))))
    grid = tuple(int(g) for g in rng.integers(8, 120, size=3))
    spacing = tuple(float(s) for s in rng.uniform(0.1, 0.6, size=3))
    nz = grid[2]
    lo = int(rng.integers(0, nz))
    band = (lo, int(rng.integers(lo + 1, nz + 1)))
    w = synth.tiny_pnn(seed=2000 + k, n=n, H=H, W=W, px=px, grid=grid,
                       tilt_deg=float(rng.uniform(0.0, 60.0)),
                       sweep_mm=float(rng.uniform(0.0, 0.6 * grid[1] * spacing[1])),
                       y0_mm=float(rng.uniform(-2.0, 0.4 * grid[1] * spacing[1])), band=band)
    origin = tuple(float(o) for o in rng.uniform(-3.0, 3.0, size=3))
    w = dataclasses.replace(w, spacing=spacing, origin=origin)
    tile = (int(rng.choice([64, 128, 256])), int(rng.integers(1, 160)), int(rng.integers(1, 9)))
    return w, tile


@pytest.mark.parametrize("k", range(24))
def test_random_geometry_bit_exact(k):
    import torch
    from paper_2412_00058_gb300 import usvol
    w, tile = random_case(k)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    imgs = torch.from_numpy(np.ascontiguousarray(w.images)).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses)).cuda()
    n, H, W = w.images.shape
    if k % 2:
        vol.set_tile(H, W, tile)
    vol.reset()
    vol.insert(imgs, poses, usvol.calibration_of(w))
    vol.fill()
    out, cnt = vol.project(*w.band)
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    g = dict(sum=acc & np.uint64(0xFFFFFFFF), cnt=(acc >> np.uint64(32)).astype(np.uint32),
             val=vol.read(usvol.READ_VALUES).cpu().numpy(),
             has=vol.read(usvol.READ_MASK).cpu().numpy(),
             proj=out.cpu().numpy(), pcnt=cnt.cpu().numpy().view(np.uint16))
    o = oracle_run(w)
    assert vol.status() == 0 and o["skipped"] == 0
    assert_pnn_bit_exact(g, o)


def random_trilinear_case(k: int):
    from paper_2412_00058_gb300 import synth
    rng = np.random.default_rng(3000 + k)
    spacing = tuple(float(s) for s in rng.uniform(0.2, 0.8, size=3))
    origin = tuple(float(o) for o in rng.uniform(-3.0, 3.0, size=3))
    tile = (256, int(rng.integers(1, 129)), int(rng.integers(1, 9)))
    if k % 3 == 2:  # linear probe, uint8 frames
        grid = tuple(int(g) for g in rng.integers(10, 90, size=3))
        w = synth.tiny_pnn(seed=4000 + k, n=int(rng.integers(1, 20)), H=int(rng.integers(3, 120)),
                           W=int(rng.integers(3, 300)), px=float(rng.uniform(0.05, 0.6)),
                           grid=grid, tilt_deg=float(rng.uniform(0.0, 40.0)),
                           sweep_mm=float(rng.uniform(0.0, 5.0)),
                           y0_mm=float(rng.uniform(0.0, 0.5 * grid[1] * spacing[1])),
                           band=(0, grid[2]))
        w = dataclasses.replace(w, mode="trilinear")
    else:           # convex fan, uint8 or float32 samples
        depth = float(rng.uniform(10.0, 50.0))
        grid = (int(rng.integers(60, 160)), int(rng.integers(20, 60)), int(rng.integers(40, 140)))
        w = synth.convex_fan(seed=4000 + k, n=int(rng.integers(1, 16)),
                             H=int(rng.integers(8, 160)), W=int(rng.integers(2, 300)),
                             depth_mm=depth, r0_mm=float(rng.uniform(0.0, 30.0)),
                             sector_deg=float(rng.uniform(10.0, 120.0)), grid=grid,
                             spacing=0.4, band=(0, grid[2]), sweep_mm=float(rng.uniform(0, 6)),
                             sway_mm=2.0, y_start_mm=float(rng.uniform(2.0, 6.0)),
                             float_frames=bool(k % 2))
    return dataclasses.replace(w, spacing=spacing, origin=origin), tile


@pytest.mark.parametrize("k", range(12))
def test_random_geometry_trilinear_within_tolerance(k):
    import torch
    from helpers import assert_trilinear_close
    from paper_2412_00058_gb300 import usvol
    w, tile = random_trilinear_case(k)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear")
    imgs = torch.from_numpy(np.ascontiguousarray(w.images)).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(w.poses)).cuda()
    n, H, W = w.images.shape
    if k % 2 == 0:
        vol.set_tile(H, W, tile)
    vol.reset()
    vol.insert(imgs, poses, usvol.calibration_of(w))
    vol.fill()
    out, cnt = vol.project(*w.band)
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy()
    g = dict(S=acc[..., 0].astype(np.float64), W=acc[..., 1].astype(np.float64),
             val=vol.read(usvol.READ_VALUES).cpu().numpy(),
             has=vol.read(usvol.READ_MASK).cpu().numpy(),
             proj=out.cpu().numpy(), pcnt=cnt.cpu().numpy().view(np.uint16), band=w.band)
    o = oracle_run(w)
    assert vol.status() == 0 and o["skipped"] == 0
    assert o["W"].sum() > 0
    assert_trilinear_close(g, o)
