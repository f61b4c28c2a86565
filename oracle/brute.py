"""Independent numpy restatements for tiny inputs (test infrastructure).

These do not use the Q31.32 quantised map of the C oracle: a pixel's world
point is computed directly in FP64 as  p = P @ K @ (u*sx, 0, v*sy, 1)  and
its voxel as floor((p - origin)/spacing + 1/2).  The two agree except for
pixels within ~1e-9 voxel of a rounding boundary; ``margin`` reports how
close each pixel came so tests can tell such pixels apart.
"""
from __future__ import annotations

import numpy as np


def pixel_voxel_coords(images_shape, poses, calib, sx, sy, spacing, origin):
    """Continuous voxel coordinates q[f, v, u, 3] in FP64."""
    n, H, W = images_shape
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)                       # [H, W]
    pts = np.stack([uu * sx, np.zeros_like(uu), vv * sy, np.ones_like(uu)], axis=-1)
    M = np.einsum("fij,jk->fik", np.asarray(poses, np.float64).reshape(n, 4, 4),
                  np.asarray(calib, np.float64).reshape(4, 4))
    world = np.einsum("fij,hwj->fhwi", M, pts)[..., :3]
    return (world - np.asarray(origin)) / np.asarray(spacing)


def pnn_brute(grid, images, poses, calib, sx, sy, spacing, origin):
    """(sum u64, cnt u32, margin f64[n,H,W], in_volume bool[n,H,W])."""
    nx, ny, nz = grid
    q = pixel_voxel_coords(images.shape, poses, calib, sx, sy, spacing, origin)
    idx = np.floor(q + 0.5).astype(np.int64)
    frac = q + 0.5 - np.floor(q + 0.5)
    margin = np.min(np.minimum(frac, 1.0 - frac), axis=-1)
    inside = ((idx[..., 0] >= 0) & (idx[..., 0] < nx) & (idx[..., 1] >= 0) &
              (idx[..., 1] < ny) & (idx[..., 2] >= 0) & (idx[..., 2] < nz))
    s = np.zeros(nz * ny * nx, dtype=np.uint64)
    c = np.zeros(nz * ny * nx, dtype=np.uint32)
    lin = (idx[..., 2] * ny + idx[..., 1]) * nx + idx[..., 0]
    np.add.at(s, lin[inside], images[inside].astype(np.uint64))
    np.add.at(c, lin[inside], np.uint32(1))
    return s.reshape(nz, ny, nx), c.reshape(nz, ny, nx), margin, inside
