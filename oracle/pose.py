"""FP64 oracle of the pose-refinement loss and its gradient (test
infrastructure, like the rest of ``oracle/``).

Forward, for frames of a linear probe:
    S, W   trilinear splat (the C oracle's ora_insert_trilinear)
    V      = S / (W + eps)
    P      = mean over the depth band of V
    L      = sum (P - T)^2
Gradient with respect to the left perturbation of each pose about its frame
centre c (p' = R(w)(p - c) + c + t; t in mm, w a rotation vector), at 0:
    dL/dt = sum_s dL/dp_s,   dL/dw = sum_s (p_s - c) x dL/dp_s,
with dL/dp_s from the adjoint of the splat (derivative of the trilinear
weights on the side selected by floor(), as the forward's cell choice).

Pinned in tests/test_pose_grad.py by central finite differences of
``loss`` itself at small steps (an independent check of the derivation).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

WMIN = 2.0 ** -20


def rodrigues(w) -> np.ndarray:
    w = np.asarray(w, np.float64)
    th = float(np.linalg.norm(w))
    if th < 1e-12:
        return np.eye(3) + np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * (Kx @ Kx)


def frame_centre(pose, calib, H, W, sx, sy) -> np.ndarray:
    x = np.array([0.5 * (W - 1) * sx, 0.0, 0.5 * (H - 1) * sy, 1.0])
    return (np.asarray(pose).reshape(4, 4) @ np.asarray(calib).reshape(4, 4) @ x)[:3]


def apply_pose_delta(poses, delta, calib, H, W, sx, sy) -> np.ndarray:
    """poses'[f] = T(t) T(c) R(w) T(-c) poses[f] for delta[f] = (t, w)."""
    poses = np.asarray(poses, np.float64).reshape(-1, 4, 4)
    out = np.empty_like(poses)
    for f in range(poses.shape[0]):
        c = frame_centre(poses[f], calib, H, W, sx, sy)
        R = rodrigues(delta[f, 3:])
        out[f] = np.eye(4)
        out[f, :3, :3] = R @ poses[f, :3, :3]
        out[f, :3, 3] = R @ (poses[f, :3, 3] - c) + c + delta[f, :3]
    return out


def forward(w, poses, band, eps, target=None):
    """(S, W, P, L) in FP64; L is None without a target."""
    S, Wt, _ = oracle.insert_trilinear(w.grid, w.images, poses, w.calibration(), w.spacing,
                                       w.origin)
    lo, hi = band
    P = (S[lo:hi] / (Wt[lo:hi] + eps)).mean(axis=0)
    L = None if target is None else float(((P - target) ** 2).sum())
    return S, Wt, P, L


def loss(w, poses, band, eps, target) -> float:
    return forward(w, poses, band, eps, target)[3]


def analytic_grad(w, poses, band, eps, target):
    """(L, grad [n, 6]) in FP64."""
    S, Wt, P, L = forward(w, poses, band, eps, target)
    lo, hi = band
    B = hi - lo
    nx, ny, nz = w.grid
    g = 2.0 * (P - target) / B                       # dL/dV per (y, x)
    den = Wt[lo:hi] + eps
    aS = g[None] / den                               # dL/dS on the band
    aW = -g[None] * S[lo:hi] / den ** 2              # dL/dW on the band
    n, H, Wd = w.images.shape
    ii, jj = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(Wd, dtype=np.float64),
                         indexing="ij")
    pts = np.stack([jj.ravel() * w.sx, np.zeros(H * Wd), ii.ravel() * w.sy, np.ones(H * Wd)])
    sp = np.asarray(w.spacing, np.float64)
    org = np.asarray(w.origin, np.float64)
    grad = np.zeros((n, 6))
    for f in range(n):
        M = np.asarray(poses[f]).reshape(4, 4) @ np.asarray(w.calib).reshape(4, 4)
        p = (M @ pts)[:3].T                          # [s, 3] world mm
        q = (p - org) / sp
        i0 = np.floor(q)
        fr = q - i0
        i0 = i0.astype(np.int64)
        I = w.images[f].reshape(-1).astype(np.float64)
        # float32 samples that are not finite or exceed 2^64 are not inserted
        # (the C oracle's sample rule), so they carry no gradient
        admit = np.abs(I) <= 2.0 ** 64
        I = np.where(admit, I, 0.0)
        dq = np.zeros_like(q)
        for c in range(8):
            cc = np.array([c & 1, (c >> 1) & 1, c >> 2])
            X = i0 + cc
            phi = np.where(cc[None, :] == 1, fr, 1.0 - fr)
            wgt = phi.prod(axis=1)
            ok = ((X[:, 0] >= 0) & (X[:, 0] < nx) & (X[:, 1] >= 0) & (X[:, 1] < ny) &
                  (X[:, 2] >= lo) & (X[:, 2] < hi) & (wgt >= WMIN) & admit)
            if not ok.any():
                continue
            Xo = X[ok]
            a = I[ok] * aS[Xo[:, 2] - lo, Xo[:, 1], Xo[:, 0]] + aW[Xo[:, 2] - lo, Xo[:, 1],
                                                                   Xo[:, 0]]
            sgn = np.where(cc == 1, 1.0, -1.0)
            ph = phi[ok]
            dq[ok, 0] += a * sgn[0] * ph[:, 1] * ph[:, 2]
            dq[ok, 1] += a * sgn[1] * ph[:, 0] * ph[:, 2]
            dq[ok, 2] += a * sgn[2] * ph[:, 0] * ph[:, 1]
        gp = dq / sp
        r = p - frame_centre(poses[f], w.calib, H, Wd, w.sx, w.sy)
        grad[f, :3] = gp.sum(axis=0)
        grad[f, 3:] = np.cross(r, gp).sum(axis=0)
    return L, grad


def fd_grad(w, poses, band, eps, target, h, frames=None, comps=range(6)):
    """Central finite differences of `loss` under apply_pose_delta."""
    n = poses.shape[0]
    frames = range(n) if frames is None else frames
    out = np.full((n, 6), np.nan)
    for f in frames:
        for k in comps:
            d = np.zeros((n, 6))
            d[f, k] = h
            lp = loss(w, apply_pose_delta(poses, d, w.calib, w.H, w.W, w.sx, w.sy), band, eps,
                      target)
            lm = loss(w, apply_pose_delta(poses, -d, w.calib, w.H, w.W, w.sx, w.sy), band, eps,
                      target)
            out[f, k] = (lp - lm) / (2 * h)
    return out
