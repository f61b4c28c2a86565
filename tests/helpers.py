"""Shared helpers for the GPU parity tests: run a workload through the CUDA
path (via the C ABI) and through the CPU oracle, and compare."""
from __future__ import annotations

import numpy as np


def build_library():
    from paper_2412_00058_gb300 import build, usvol
    build.build()
    if usvol.CHECKED:
        build.build(checked=True)
    import oracle
    oracle.build()


def gpu_run(w, splits=None, band=None, dev="cuda", images=None, poses=None):
    """Insert (optionally in several calls of the given sizes), fill, project."""
    import torch
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume(w.grid, w.spacing, w.origin, w.mode, device=dev)
    vol.reset()
    imgs = torch.from_numpy(np.ascontiguousarray(w.images if images is None else images)).to(dev)
    ps = torch.from_numpy(np.ascontiguousarray(w.poses if poses is None else poses)).to(dev)
    cal = usvol.calibration_of(w)
    if splits is None:
        splits = [imgs.shape[0]]
    f = 0
    for k in splits:
        vol.insert(imgs[f:f + k], ps[f:f + k], cal)
        f += k
    assert f == imgs.shape[0]
    vol.fill()
    lo, hi = band or w.band
    out, cnt = vol.project(lo, hi)
    st = vol.status()
    res = dict(status=st, vol=vol, band=(lo, hi))
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy()
    if w.mode == "pnn" or w.mode == 0:
        acc = acc.view(np.uint64)
        res["sum"] = acc & np.uint64(0xFFFFFFFF)
        res["cnt"] = (acc >> np.uint64(32)).astype(np.uint32)
    else:
        res["S"] = acc[..., 0].astype(np.float64)
        res["W"] = acc[..., 1].astype(np.float64)
    res["val"] = vol.read(usvol.READ_VALUES).cpu().numpy()
    res["has"] = vol.read(usvol.READ_MASK).cpu().numpy()
    res["proj"] = out.cpu().numpy()
    res["pcnt"] = cnt.cpu().numpy().view(np.uint16)
    return res


def oracle_run(w, band=None, images=None, poses=None):
    import oracle
    imgs = w.images if images is None else images
    ps = w.poses if poses is None else poses
    lo, hi = band or w.band
    if w.mode == "pnn":
        s, c, sk = oracle.insert_pnn(w.grid, imgs, ps, w.calib, w.sx, w.sy, w.spacing, w.origin)
        val, has = oracle.fill_pnn(s, c)
        proj, pcnt = oracle.project_u8(val, has, lo, hi)
        return dict(sum=s, cnt=c, val=val, has=has, proj=proj, pcnt=pcnt, skipped=sk)
    S, Wt, sk = oracle.insert_trilinear(w.grid, imgs, ps, w.calibration(), w.spacing, w.origin)
    val, has = oracle.fill_trilinear(S, Wt)
    proj, pcnt = oracle.project_f64(val, has, lo, hi)
    return dict(S=S, W=Wt, val=val, has=has, proj=proj, pcnt=pcnt, skipped=sk)


def assert_pnn_bit_exact(g, o):
    assert np.array_equal(g["cnt"], o["cnt"]), f"counts differ at {np.argwhere(g['cnt'] != o['cnt'])[:5]}"
    assert np.array_equal(g["sum"], o["sum"]), f"sums differ at {np.argwhere(g['sum'] != o['sum'])[:5]}"
    assert np.array_equal(g["has"], o["has"]), "has-data mask differs"
    assert np.array_equal(g["val"], o["val"]), f"values differ at {np.argwhere(g['val'] != o['val'])[:5]}"
    assert np.array_equal(g["pcnt"], o["pcnt"]), "projection counts differ"
    assert np.array_equal(g["proj"], o["proj"]), "projection differs"


# Tolerance for the FP32 weighted path against the FP64 oracle:
#   |g - o| <= RTOL*|o| + ATOL_FRAC*max|o|, skipping voxels whose oracle
#   weight is below 2^-18 (where the 2^-20 weight cut-off dominates).
RTOL = 1e-5
ATOL_FRAC = 1e-6
WSKIP = 2.0 ** -18


def close(g, o, rtol=RTOL, atol_frac=ATOL_FRAC, mask=None):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    if mask is not None:
        g, o = g[mask], o[mask]
    if o.size == 0:
        return True, 0.0
    tol = rtol * np.abs(o) + atol_frac * np.abs(o).max()
    err = np.abs(g - o)
    worst = float(np.max(err / np.maximum(tol, 1e-300)))
    return bool(np.all(err <= tol)), worst


def effective_weight(W):
    """A voxel's own weight, or for an empty voxel the pooled weight of its
    26 neighbours (what its filled value is divided by)."""
    from scipy.ndimage import convolve
    k = np.ones((3, 3, 3))
    k[1, 1, 1] = 0.0
    pooled = convolve(W, k, mode="constant", cval=0.0)
    return np.where(W > 0, W, pooled)


def assert_trilinear_close(g, o):
    keep = o["W"] >= WSKIP
    for k in ("S", "W"):
        ok, worst = close(g[k], o[k], mask=keep)
        assert ok, f"{k}: worst error / tolerance = {worst:.3g}"
    # empty iff W == 0 on both sides, except where the 2^-20 cut-off decides
    strong = (o["W"] >= WSKIP) | (o["W"] == 0)
    assert np.array_equal((g["W"] > 0)[strong], (o["W"] > 0)[strong])
    weff = effective_weight(o["W"])
    decided = (weff >= WSKIP) | (weff == 0)
    assert np.array_equal(g["has"][decided], o["has"][decided])
    both = (g["has"] == 1) & (o["has"] == 1) & (weff >= WSKIP)
    ok, worst = close(g["val"], o["val"], mask=both)
    assert ok, f"values: worst error / tolerance = {worst:.3g}"
    # projection: columns whose band holds only well-decided voxels
    lo, hi = g.get("band", (None, None))
    weak = (o["has"] == 1) & (weff < WSKIP)
    cols = ~weak[lo:hi].any(axis=0) if lo is not None else np.ones(o["proj"].shape, bool)
    ok, worst = close(g["proj"], o["proj"], mask=cols)
    assert ok, f"projection: worst error / tolerance = {worst:.3g}"
    assert cols.mean() > 0.99
