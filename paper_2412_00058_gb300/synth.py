"""Seeded synthetic inputs for the free-hand ultrasound volume path.

This module only *makes inputs*: B-mode frames, probe->world poses and the
probe calibration.  It holds none of the reconstruction arithmetic (no
pixel->voxel mapping, no accumulation, no hole filling, no projection), so
both the CPU oracle and the CUDA path can be fed from it without sharing any
of the method's code.

Workloads follow the scan the paper describes: a free-hand sweep over the
whole spine (shoulder to crotch, > 500 mm) in about 2 minutes at 30 fps
(Sec. III.B), an operator scanning side by side columns (Sec. II.C), bone
surfaces that appear as bright arcs with an acoustic shadow underneath
(Sec. II.D, discussion of Algorithm 2).  The patient data itself is not
public; Rayleigh speckle plus bright arcs stands in for it.

Axis convention: x lateral, y along the spine (sweep direction), z depth.
A linear-probe frame pixel (u, v) (column u, row v) sits at the image-frame
point (u*sx, 0, v*sy) mm; ``calib`` maps the image frame to the probe frame
and ``poses[f]`` maps the probe frame to the world frame (the paper's
T_T^W).  All matrices are 4x4 row-major float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 2412_00058


@dataclass
class Workload:
    name: str
    images: np.ndarray            # [n, H, W] uint8 (or float32)
    poses: np.ndarray             # [n, 4, 4] float64, probe -> world
    calib: np.ndarray             # [4, 4] float64, image -> probe
    grid: tuple                   # (nx, ny, nz)
    spacing: tuple                # voxel spacing (mm) per axis
    origin: tuple                 # centre of voxel (0,0,0) in mm
    band: tuple                   # (z_lo, z_hi) half-open voxel rows
    mode: str = "pnn"             # "pnn" | "trilinear"
    geom: str = "linear"          # "linear" | "convex"
    sx: float = 0.0               # linear: lateral pixel spacing (mm)
    sy: float = 0.0               # linear: axial pixel spacing (mm)
    r0: float = 0.0               # convex: radius of the first sample (mm)
    dr: float = 0.0               # convex: radial sample spacing (mm)
    sector_deg: float = 0.0       # convex: full sector angle
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.images.shape[0])

    @property
    def H(self) -> int:
        return int(self.images.shape[1])

    @property
    def W(self) -> int:
        return int(self.images.shape[2])

    def calibration(self) -> dict:
        return dict(image_to_probe=self.calib, sx=self.sx, sy=self.sy,
                    geom=self.geom, r0=self.r0, dr=self.dr,
                    sector_deg=self.sector_deg)


# ----------------------------------------------------------------------------
# small matrix helpers (input construction only)
# ----------------------------------------------------------------------------

def rot_x(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def rot_y(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def rigid(R: np.ndarray, t) -> np.ndarray:
    T = np.eye(4, dtype=np.float64)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(t, dtype=np.float64)
    return T


def translation(t) -> np.ndarray:
    return rigid(np.eye(3), t)


# ----------------------------------------------------------------------------
# speckle and anatomy
# ----------------------------------------------------------------------------

def rayleigh_u8(rng: np.random.Generator, shape, sigma: float = 40.0) -> np.ndarray:
    """min(255, round(Rayleigh(sigma))) as uint8."""
    x = rng.rayleigh(scale=sigma, size=shape)
    return np.minimum(np.rint(x), 255.0).astype(np.uint8)


class _SpeckleBank:
    """A bank of independent Rayleigh speckle frames; frame f takes bank entry
    f mod B, circularly shifted by a seeded offset, so that a 3600-frame sweep
    is generated in seconds instead of sampling 10^9 Rayleigh variates."""

    def __init__(self, rng: np.random.Generator, H: int, W: int, count: int = 24,
                 sigma: float = 40.0):
        self.bank = rayleigh_u8(rng, (count, H, W), sigma)
        self.rng = rng

    def frame(self, f: int) -> np.ndarray:
        b = self.bank[f % self.bank.shape[0]]
        dv = int(self.rng.integers(0, b.shape[0]))
        du = int(self.rng.integers(0, b.shape[1]))
        return np.roll(np.roll(b, dv, axis=0), du, axis=1)


def _draw_bone(img: np.ndarray, rows_centre: np.ndarray, half_rows: float,
               rng: np.random.Generator, shadow: float = 0.2) -> None:
    """Bright cortical arc (220..255) centred on rows_centre[u] (one value per
    column), +-half_rows thick, with the acoustic shadow underneath scaled by
    ``shadow`` (bone does not transmit ultrasound, Sec. II.D)."""
    H, W = img.shape
    v = np.arange(H, dtype=np.float64)[:, None]
    c = rows_centre[None, :]
    arc = np.abs(v - c) <= half_rows
    below = v > c + half_rows
    img[below] = (img[below].astype(np.float32) * shadow).astype(np.uint8)
    vals = rng.integers(220, 256, size=int(arc.sum()), dtype=np.int64)
    img[arc] = vals.astype(np.uint8)


# ----------------------------------------------------------------------------
# workload 1: tiny PNN reconstruction
# ----------------------------------------------------------------------------

def tiny_pnn(seed: int = SEED_BASE + 0, n: int = 64, H: int = 128, W: int = 128,
             px: float = 0.3, grid=(128, 128, 128), spacing: float = 0.3,
             band=(60, 80), tilt_deg: float = 2.0, sweep_mm: float = 20.0,
             y0_mm: float = 9.2) -> Workload:
    """64 frames of 128x128 uint8 speckle (sigma 40) with one bright arc at
    about 40 px depth; 0.3 mm pixels; a straight 20 mm sweep along y with
    seeded +-2 deg tilts about x, y and z around the frame centre; a 128^3
    volume at 0.3 mm; depth band [60, 80)."""
    rng = np.random.default_rng(seed)
    imgs = rayleigh_u8(rng, (n, H, W))
    u = np.arange(W, dtype=np.float64)
    arc_rows = 40.0 + 0.002 * (u - W / 2) ** 2
    v = np.arange(H, dtype=np.float64)[:, None]
    mask = np.abs(v - arc_rows[None, :]) <= 1.0
    imgs[:, mask] = 230
    poses = np.empty((n, 4, 4), dtype=np.float64)
    t = math.radians(tilt_deg)
    for f in range(n):
        y = y0_mm + sweep_mm * f / max(n - 1, 1)
        ax, ay, az = rng.uniform(-t, t, size=3)
        R = rot_z(az) @ rot_y(ay) @ rot_x(ax)
        c = np.array([(W - 1) * px / 2, y, (H - 1) * px / 2])
        # untilted: image (x, 0, z) -> (x, y, z); tilt about the frame centre c
        poses[f] = rigid(R, c + R @ (np.array([0.0, y, 0.0]) - c))
    return Workload("tiny_pnn", imgs, poses, np.eye(4), tuple(grid),
                    (spacing,) * 3, (0.0, 0.0, 0.0), tuple(band),
                    sx=px, sy=px, meta=dict(seed=seed))


# ----------------------------------------------------------------------------
# workload 2: whole-spine linear-probe sweep
# ----------------------------------------------------------------------------

def whole_spine(seed: int = SEED_BASE + 1, n: int = 3600, H: int = 640, W: int = 480,
                aperture_mm=(40.0, 60.0), sweep_mm: float = 550.0,
                grid=(270, 1840, 200), spacing: float = 0.3, band=(117, 150),
                sway_mm: float = 20.0, tilt_deg: float = 10.0,
                jitter_deg: float = 1.0, y_start_mm: float = 0.0,
                y_span_mm: float | None = None) -> Workload:
    """Whole-spine sweep: n frames (2 min at 30 fps = 3600) of H x W uint8
    speckle (W lateral columns over 40 mm, H depth rows over 60 mm) with a
    1 mm bone arc at depth 45 + 15 sin(2 pi y / 550) mm (30..60 mm) and its
    shadow; probe path 550 mm along y with a +-20 mm lateral sway (three
    sways, echoing the three side-by-side columns of Sec. II.C), in-plane
    tilt 10 deg * sin(2 pi y / 137) plus +-1 deg seeded jitter about x and z;
    volume 270 x 1840 x 200 at 0.3 mm; band [117, 150) = 35..45 mm, the two
    fixed VPI depths of Sec. III.B.

    ``y_start_mm``/``y_span_mm`` cut a short piece of the same sweep (used for
    scaled-down parity cases) while keeping its local geometry."""
    rng = np.random.default_rng(seed)
    sx = aperture_mm[0] / W
    sy = aperture_mm[1] / H
    span = sweep_mm if y_span_mm is None else y_span_mm
    bank = _SpeckleBank(rng, H, W)
    imgs = np.empty((n, H, W), dtype=np.uint8)
    poses = np.empty((n, 4, 4), dtype=np.float64)
    calib = translation([-(W - 1) * sx / 2.0, 0.0, 0.0])  # probe origin: top centre
    lat = (np.arange(W, dtype=np.float64) - (W - 1) / 2.0) * sx
    jit = math.radians(jitter_deg)
    for f in range(n):
        y = y_start_mm + span * f / max(n - 1, 1)
        x = grid[0] * spacing / 2.0 + sway_mm * math.sin(2 * math.pi * y / 183.0)
        tilt = math.radians(tilt_deg) * math.sin(2 * math.pi * y / 137.0)
        jx, jz = rng.uniform(-jit, jit, size=2)
        R = rot_y(tilt) @ rot_x(jx) @ rot_z(jz)
        poses[f] = rigid(R, [x, y, 0.0])
        img = bank.frame(f)
        depth = 45.0 + 15.0 * math.sin(2 * math.pi * y / 550.0)
        rows = (depth - 4.0 * (1.0 - (lat / (aperture_mm[0] / 2)) ** 2)) / sy
        _draw_bone(img, rows, 0.5 / sy, rng)
        imgs[f] = img
    return Workload("whole_spine", imgs, poses, calib, tuple(grid), (spacing,) * 3,
                    (0.0, 0.0, 0.0), tuple(band), sx=sx, sy=sy,
                    meta=dict(seed=seed, sweep_mm=span))


# ----------------------------------------------------------------------------
# workload 3: convex-probe fan, trilinear splatting
# ----------------------------------------------------------------------------

def convex_fan(seed: int = SEED_BASE + 2, n: int = 3000, H: int = 512, W: int = 512,
               depth_mm: float = 120.0, r0_mm: float = 40.0, sector_deg: float = 60.0,
               grid=(400, 1700, 400), spacing: float = 0.4, band=(87, 113),
               sweep_mm: float = 660.0, sway_mm: float = 20.0,
               tilt_deg: float = 10.0, jitter_deg: float = 1.0,
               y_start_mm: float = 4.0, float_frames: bool = False) -> Workload:
    """Convex probe (the paper's system uses a 6C1 convex array, Sec. III.A):
    n pre-scan-conversion polar frames, row i = radial sample at
    r = r0 + i*dr (dr = depth/(H-1)), column j = beam at angle
    -sector/2 + j*sector/(W-1).  The in-plane point of sample (i, j) is
    (r sin(theta), 0, r cos(theta) - r0) in the probe frame (origin at the
    centre of the transducer face).  Volume 400 x 1700 x 400 at 0.4 mm."""
    rng = np.random.default_rng(seed)
    dr = depth_mm / (H - 1)
    bank = _SpeckleBank(rng, H, W)
    imgs = np.empty((n, H, W), dtype=np.float32 if float_frames else np.uint8)
    poses = np.empty((n, 4, 4), dtype=np.float64)
    jit = math.radians(jitter_deg)
    half = math.radians(sector_deg) / 2.0
    z0 = r0_mm * (1.0 - math.cos(half)) + 0.5
    theta = -half + np.arange(W, dtype=np.float64) * (2 * half / (W - 1))
    for f in range(n):
        y = y_start_mm + sweep_mm * f / max(n - 1, 1)
        x = grid[0] * spacing / 2.0 + sway_mm * math.sin(2 * math.pi * y / 226.0)
        tilt = math.radians(tilt_deg) * math.sin(2 * math.pi * y / 169.0)
        jx, jz = rng.uniform(-jit, jit, size=2)
        R = rot_y(tilt) @ rot_x(jx) @ rot_z(jz)
        poses[f] = rigid(R, [x, y, z0])
        img = bank.frame(f)
        depth = 55.0 + 15.0 * math.sin(2 * math.pi * y / 680.0)
        # bone at constant depth below the skin: radius where r cos(theta) - r0 = depth
        rows = ((depth + r0_mm) / np.cos(theta) - r0_mm) / dr
        _draw_bone(img, rows, 0.5 / dr, rng)
        imgs[f] = img.astype(imgs.dtype)
    return Workload("convex_fan", imgs, poses, np.eye(4), tuple(grid), (spacing,) * 3,
                    (0.0, 0.0, 0.0), tuple(band), mode="trilinear", geom="convex",
                    r0=r0_mm, dr=dr, sector_deg=sector_deg, meta=dict(seed=seed))


# ----------------------------------------------------------------------------
# workload 5: differentiable pose refinement (FP32 frames, trilinear)
# ----------------------------------------------------------------------------

def pose_refine(seed: int = SEED_BASE + 4, n: int = 512, H: int = 256, W: int = 256,
                px: float = 0.2, grid=(256, 512, 192), spacing: float = 0.3,
                band=(80, 140), sweep_mm: float = 120.0, trans_sigma_mm: float = 1.0,
                rot_sigma_deg: float = 1.0) -> Workload:
    """512 FP32 frames of 256x256 at 0.2 mm/px, a 120 mm sweep into a
    256 x 512 x 192 volume at 0.3 mm; ground-truth poses plus seeded
    perturbations N(0, 1 mm) (translation) and N(0, 1 deg) (rotation) kept
    in ``meta['noisy_poses']``."""
    rng = np.random.default_rng(seed)
    imgs = rayleigh_u8(rng, (n, H, W)).astype(np.float32)
    u = np.arange(W, dtype=np.float64)
    rows = 150.0 + 0.004 * (u - W / 2) ** 2
    v = np.arange(H, dtype=np.float64)[:, None]
    imgs[:, np.abs(v - rows[None, :]) <= 2.0] = 240.0
    calib = translation([-(W - 1) * px / 2.0, 0.0, 0.0])
    poses = np.empty((n, 4, 4), dtype=np.float64)
    noisy = np.empty_like(poses)
    for f in range(n):
        y = 16.0 + sweep_mm * f / max(n - 1, 1)
        x = grid[0] * spacing / 2.0 + 5.0 * math.sin(2 * math.pi * y / 90.0)
        R = rot_y(math.radians(5.0) * math.sin(2 * math.pi * y / 70.0))
        poses[f] = rigid(R, [x, y, 2.0])
        dt = rng.normal(0.0, trans_sigma_mm, size=3)
        da = np.radians(rng.normal(0.0, rot_sigma_deg, size=3))
        dR = rot_z(da[2]) @ rot_y(da[1]) @ rot_x(da[0])
        noisy[f] = rigid(dR @ R, poses[f, :3, 3] + dt)
    return Workload("pose_refine", imgs, poses, calib, tuple(grid), (spacing,) * 3,
                    (0.0, 0.0, 0.0), tuple(band), mode="trilinear", sx=px, sy=px,
                    meta=dict(seed=seed, noisy_poses=noisy))


# ----------------------------------------------------------------------------
# workload 4: concurrent streaming sessions
# ----------------------------------------------------------------------------

def streaming_sessions(seconds: float = 4.0, seed: int = SEED_BASE + 3):
    """Four concurrent scans (name, workload, frames per second): a 128^3
    volume at 30 fps, a 256 x 1024 x 200 spine piece at 60 fps, the whole
    spine 270 x 1840 x 200 at 120 fps and the 400 x 1700 x 400 convex fan
    (trilinear) at 30 fps, each with enough frames for `seconds` of scan."""
    out = []
    n1 = max(2, int(30 * seconds) + 1)
    out.append(("tiny_128", tiny_pnn(seed=seed, n=n1, sweep_mm=20.0), 30.0))
    n2 = max(2, int(60 * seconds) + 1)
    out.append(("spine_256x1024x200",
                whole_spine(seed=seed + 1, n=n2, grid=(256, 1024, 200),
                            y_start_mm=10.0, y_span_mm=min(280.0, n2 * 550.0 / 3599.0)), 60.0))
    n3 = max(2, int(120 * seconds) + 1)
    out.append(("spine_270x1840x200",
                whole_spine(seed=seed + 2, n=n3, y_span_mm=min(550.0, n3 * 550.0 / 3599.0)),
                120.0))
    n4 = max(2, int(30 * seconds) + 1)
    out.append(("convex_400x1700x400",
                convex_fan(seed=seed + 3, n=n4, sweep_mm=min(660.0, n4 * 660.0 / 2999.0)), 30.0))
    return out
