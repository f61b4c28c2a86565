"""Streaming sessions (incremental insertion with region refresh, Sec. II.C):
admission by device memory on the CPU; on the GPU, a streamed scan must
leave exactly the volume of a one-shot insertion, and its region-refreshed
projection must equal a full fill + projection of that volume."""
import numpy as np
import pytest


def test_admission_refuses_sessions_over_the_memory_budget():
    from paper_2412_00058_gb300 import stream, synth, usvol
    usvol.lib()
    w = synth.tiny_pnn(n=4, H=16, W=16)
    need = stream.session_bytes(w)
    sched = stream.Scheduler.__new__(stream.Scheduler)
    sched.device, sched.budget, sched.used, sched.sessions = None, need - 1, 0, []
    with pytest.raises(stream.AdmissionError):
        sched.admit("too_big", w, 30.0)
    assert sched.used == 0 and sched.sessions == []


def test_frames_voxel_box_contains_every_pixel_voxel():
    from paper_2412_00058_gb300 import stream, synth
    from oracle import brute
    w = synth.whole_spine(n=5, grid=(270, 60, 200), y_start_mm=3.0, y_span_mm=5.0)
    lo, hi = stream.frames_voxel_box(w, w.poses, margin=0)
    q = brute.pixel_voxel_coords(w.images.shape, w.poses, w.calib, w.sx, w.sy, w.spacing,
                                 w.origin)
    idx = np.floor(q + 0.5).astype(np.int64).reshape(-1, 3)
    n = np.asarray(w.grid)
    inside = np.all((idx >= 0) & (idx < n), axis=1)
    assert np.all(idx[inside] >= lo) and np.all(idx[inside] < hi)


@pytest.mark.gpu
@pytest.mark.parametrize("batched,realtime", [(False, True), (True, True), (True, False)])
def test_streamed_scan_equals_one_shot_and_full_refresh(batched, realtime):
    """Per-session streams, and the batched engine (one multi-volume
    insertion per dispatch over two nearest-neighbour sessions and a
    trilinear one), paced in real time or replayed at once."""
    import torch
    from helpers import build_library
    from paper_2412_00058_gb300 import stream, synth, usvol
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()
    sched = stream.Scheduler("cuda")
    w1 = synth.whole_spine(n=90, grid=(270, 200, 200), y_start_mm=5.0, y_span_mm=14.0)
    w2 = synth.convex_fan(n=40, H=160, W=96, depth_mm=40.0, r0_mm=20.0, grid=(180, 80, 150),
                          spacing=0.4, band=(40, 70), sweep_mm=12.0, sway_mm=3.0,
                          y_start_mm=6.0)
    w3 = synth.tiny_pnn(n=50)
    s1 = sched.admit("pnn", w1, 120.0, seed=1)
    s2 = sched.admit("tri", w2, 60.0, seed=2)
    s3 = sched.admit("tiny", w3, 60.0, seed=3)
    stats = sched.run(batched=batched, realtime=realtime)
    torch.cuda.synchronize()
    assert [st.frames for st in stats] == [w1.n, w2.n, w3.n]
    summ = stream.summary(stats)
    if realtime:
        assert summ["p99_ms"] < 100.0
    if batched:
        assert sched.dispatches <= sum(st.bursts for st in stats)
    for s, w in ((s1, w1), (s2, w2), (s3, w3)):
        ref = usvol.Volume(w.grid, w.spacing, w.origin, w.mode)
        ref.reset()
        ref.insert(torch.from_numpy(w.images).cuda(), torch.from_numpy(w.poses).cuda(),
                   usvol.calibration_of(w))
        if w.mode == "pnn":       # integer accumulation: any batching gives the same bytes
            assert torch.equal(s.vol.read(usvol.READ_ACCUM), ref.read(usvol.READ_ACCUM))
        # the incrementally refreshed image equals a full refresh of the streamed volume
        s.vol.fill()
        full, fcnt = s.vol.project(*w.band)
        torch.cuda.synchronize()
        assert torch.equal(s.out, full) and torch.equal(s.cnt, fcnt)
