"""Hand-worked examples (tests/golden/*.txt, each citing the passages its
values follow): the oracle on the CPU and the CUDA path through the C ABI
must both reproduce every value -- the nearest-neighbour path bit for bit,
the trilinear one exactly as well (all its weights are powers of two)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    """key = numbers, rows separated by '/'; '#' starts a comment."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            rows = [[float(x) for x in r.split()] for r in val.split("/")]
            if len(rows) == 1 and len(rows[0]) == 1:
                out[key] = rows[0][0]
            else:
                out[key] = np.array(rows if len(rows) > 1 else rows[0])
    return out


def pnn_case():
    g = read_fixture("pnn_worked_example.txt")
    grid = tuple(int(x) for x in g["grid"])
    images = np.stack([g["frame0"], g["frame1"]]).astype(np.uint8)
    pose = np.eye(4)
    pose[:3, 3] = g["translation_mm"]
    poses = np.stack([pose, pose])
    nx, ny, nz = grid
    s = np.zeros((nz, ny, nx), np.uint64)
    c = np.zeros((nz, ny, nx), np.uint32)
    s[:2, 1, :3] = g["sum_y1"]
    c[:2, 1, :3] = g["count_y1"]
    val = np.stack([g["value_z0"], g["value_z1"], g["value_z2"]]).astype(np.uint8)
    lo, hi = (int(x) for x in g["band"])
    proj = g["proj_sum"].astype(np.float32) / np.float32(hi - lo)
    return dict(grid=grid, images=images, poses=poses, spacing=tuple(g["spacing_mm"]),
                origin=tuple(g["origin_mm"]), sx=g["pixel_mm"][0], sy=g["pixel_mm"][1],
                sum=s, cnt=c, val=val, has=np.ones_like(val), band=(lo, hi), proj=proj,
                pcnt=g["proj_count"].astype(np.uint16))


def trilinear_case():
    g = read_fixture("trilinear_worked_example.txt")
    grid = tuple(int(x) for x in g["grid"])
    nx, ny, nz = grid
    pose = np.eye(4)
    pose[:3, 3] = g["translation_mm"]
    S = np.zeros((nz, ny, nx))
    W = np.zeros((nz, ny, nx))
    S[:2, :2, :2] = float(g["cell_S"])
    W[:2, :2, :2] = float(g["cell_W"])
    e = int(g["filled_extent"])
    val = np.zeros((nz, ny, nx))
    has = np.zeros((nz, ny, nx), np.uint8)
    val[:e, :e, :e] = float(g["filled_value"])
    has[:e, :e, :e] = 1
    proj = np.zeros((ny, nx))
    pcnt = np.zeros((ny, nx), np.uint16)
    proj[:e, :e] = float(g["proj_value"])
    pcnt[:e, :e] = int(g["proj_count"])
    lo, hi = (int(x) for x in g["band"])
    return dict(grid=grid, images=np.full((1, 1, 1), int(g["intensity"]), np.uint8),
                poses=pose[None], spacing=tuple(g["spacing_mm"]), origin=tuple(g["origin_mm"]),
                sx=g["pixel_mm"][0], sy=g["pixel_mm"][1], S=S, W=W, val=val, has=has,
                band=(lo, hi), proj=proj, pcnt=pcnt)


def test_fixtures_are_self_consistent():
    """The hand-written values agree with each other: counts sum to the
    pixels, the projection sums are the column sums of the filled values."""
    p = pnn_case()
    assert int(p["cnt"].sum()) == p["images"].size
    assert int(p["sum"].sum()) == int(p["images"].astype(np.int64).sum())
    lo, hi = p["band"]
    assert np.array_equal(p["val"][lo:hi].astype(np.int64).sum(axis=0),
                          (p["proj"] * np.float32(hi - lo)).round().astype(np.int64))
    t = trilinear_case()
    assert t["W"].sum() == 1.0 and t["S"].sum() == float(t["images"][0, 0, 0])


def test_oracle_reproduces_the_pnn_example():
    import oracle
    oracle.build()
    p = pnn_case()
    s, c, skipped = oracle.insert_pnn(p["grid"], p["images"], p["poses"], np.eye(4), p["sx"],
                                      p["sy"], p["spacing"], p["origin"])
    assert skipped == 0
    assert np.array_equal(s, p["sum"]) and np.array_equal(c, p["cnt"])
    val, has = oracle.fill_pnn(s, c)
    assert np.array_equal(val, p["val"]) and np.array_equal(has, p["has"])
    proj, pcnt = oracle.project_u8(val, has, *p["band"])
    assert np.array_equal(proj, p["proj"]) and np.array_equal(pcnt, p["pcnt"])


def test_oracle_reproduces_the_trilinear_example():
    import oracle
    oracle.build()
    t = trilinear_case()
    cal = dict(image_to_probe=np.eye(4), sx=t["sx"], sy=t["sy"], geom="linear", r0=0.0,
               dr=0.0, sector_deg=0.0)
    S, W, skipped = oracle.insert_trilinear(t["grid"], t["images"], t["poses"], cal,
                                            t["spacing"], t["origin"])
    assert skipped == 0
    assert np.array_equal(S, t["S"]) and np.array_equal(W, t["W"])
    val, has = oracle.fill_trilinear(S, W)
    assert np.array_equal(has, t["has"]) and np.array_equal(val[has == 1], t["val"][has == 1])
    proj, pcnt = oracle.project_f64(val, has, *t["band"])
    assert np.array_equal(proj, t["proj"]) and np.array_equal(pcnt, t["pcnt"])


def _gpu_volume(case, mode):
    import torch
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume(case["grid"], case["spacing"], case["origin"], mode)
    vol.reset()
    imgs = torch.from_numpy(np.ascontiguousarray(case["images"])).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(case["poses"])).cuda()
    vol.insert(imgs, poses, usvol.make_calibration(np.eye(4), "linear", case["sx"], case["sy"]))
    vol.fill()
    out, cnt = vol.project(*case["band"])
    assert vol.status() == 0
    return vol, out.cpu().numpy(), cnt.cpu().numpy().view(np.uint16)


@pytest.mark.gpu
def test_cuda_path_reproduces_the_pnn_example():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from helpers import build_library
    from paper_2412_00058_gb300 import usvol
    build_library()
    p = pnn_case()
    vol, out, cnt = _gpu_volume(p, "pnn")
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)
    assert np.array_equal(acc & np.uint64(0xFFFFFFFF), p["sum"])
    assert np.array_equal(acc >> np.uint64(32), p["cnt"].astype(np.uint64))
    assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), p["val"])
    assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), p["has"])
    assert np.array_equal(out, p["proj"]) and np.array_equal(cnt, p["pcnt"])


@pytest.mark.gpu
def test_cuda_path_reproduces_the_trilinear_example():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from helpers import build_library
    from paper_2412_00058_gb300 import usvol
    build_library()
    t = trilinear_case()
    vol, out, cnt = _gpu_volume(t, "trilinear")
    acc = vol.read(usvol.READ_ACCUM).cpu().numpy()
    assert np.array_equal(acc[..., 0], t["S"].astype(np.float32))
    assert np.array_equal(acc[..., 1], t["W"].astype(np.float32))
    has = vol.read(usvol.READ_MASK).cpu().numpy()
    assert np.array_equal(has, t["has"])
    val = vol.read(usvol.READ_VALUES).cpu().numpy()
    assert np.array_equal(val[has == 1], t["val"][has == 1].astype(np.float32))
    assert np.array_equal(out, t["proj"].astype(np.float32)) and np.array_equal(cnt, t["pcnt"])
