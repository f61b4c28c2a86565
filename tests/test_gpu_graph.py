"""The library's calls inside a captured CUDA graph: a sweep step (insert,
fill with in-pass clearing, projection) captured twice -- the two
accumulator sets swap at every step -- and replayed gives, replay after
replay, exactly the CPU oracle's filled volume and projection (and the eager
GPU results).  Host-pose insertion refuses to be captured."""
import numpy as np
import pytest

from helpers import build_library, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def test_sweep_step_replays_from_a_cuda_graph():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.whole_spine(n=47, grid=(270, 90, 200), y_start_mm=3.0, y_span_mm=20.0)
    imgs = torch.from_numpy(w.images).cuda()
    poses = torch.from_numpy(w.poses).cuda()
    cal = usvol.calibration_of(w)
    lo, hi = w.band
    ny, nx = w.grid[1], w.grid[0]

    ref = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    ref.reset()
    ref.insert(imgs, poses, cal)
    ref.fill()
    want_out, want_cnt = ref.project(lo, hi)
    want_val = ref.read(usvol.READ_VALUES)

    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn", spare=True)
    out = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    cnt = torch.empty((ny, nx), dtype=torch.int16, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):   # warm-up: first-use set-up happens outside capture
        vol.reset()
        for _ in range(2):
            vol.insert(imgs, poses, cal)
            vol.fill_and_clear()
            vol.project(lo, hi, out=out, count=cnt)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(2):
            vol.insert(imgs, poses, cal)
            vol.fill_and_clear()
            vol.project(lo, hi, out=out, count=cnt)
    o = oracle_run(w)
    assert np.array_equal(want_out.cpu().numpy(), o["proj"])
    for _ in range(3):
        out.zero_()
        cnt.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), o["proj"])
        assert np.array_equal(cnt.cpu().numpy().view(np.uint16), o["pcnt"])
        assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), o["val"])
        assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), o["has"])
        assert torch.equal(out, want_out) and torch.equal(cnt, want_cnt)
        assert torch.equal(vol.read(usvol.READ_VALUES), want_val)
        assert not vol.read(usvol.READ_ACCUM).any()
    assert vol.status() == 0


def test_host_pose_insert_is_refused_inside_a_capture():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=4, H=16, W=16)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    imgs = torch.from_numpy(w.images).cuda()
    cal = usvol.calibration_of(w)
    vol.reset()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=side):
        try:
            vol.insert(imgs, w.poses, cal)      # host poses
        except usvol.UsvError as e:
            err = e
    assert err is not None and err.code == usvol.ERR_UNSUPPORTED
