"""Streaming sessions (incremental insertion with region refresh, Sec. II.C):
admission by device memory and the library's region box on the CPU; on the
GPU, a streamed scan's volume and its region-refreshed projection against
the CPU oracle of all its frames (bit-exact for nearest neighbour, within
the trilinear tolerance for the weighted session), and against a full fill
+ projection of the streamed volume itself."""
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


def _box(w, poses, margin=0):
    from paper_2412_00058_gb300 import usvol
    p = np.ascontiguousarray(poses, np.float64)
    return usvol.frames_voxel_box(w.grid, w.spacing, w.origin, p.ctypes.data, p.shape[0], w.H,
                                  w.W, usvol.calibration_of(w), margin)


def test_frames_voxel_box_contains_every_voxel_written():
    """usv_frames_voxel_box (host code in the library, no GPU needed) holds
    every voxel the oracle writes -- nearest voxels for PNN, all corners with
    weight for trilinear, linear and convex -- and is at most a few voxels
    larger than their bounding box (a linear probe)."""
    import oracle
    from paper_2412_00058_gb300 import synth
    cases = [synth.whole_spine(n=5, grid=(270, 60, 200), y_start_mm=3.0, y_span_mm=5.0),
             synth.convex_fan(n=4, H=64, W=48, depth_mm=30.0, r0_mm=20.0, grid=(160, 60, 120),
                              spacing=0.4, band=(20, 40), sweep_mm=3.0, sway_mm=2.0,
                              y_start_mm=8.0)]
    for w in cases:
        if w.mode == "pnn":
            _, c, _ = oracle.insert_pnn(w.grid, w.images, w.poses, w.calib, w.sx, w.sy,
                                        w.spacing, w.origin)
            hit = c > 0
        else:
            _, Wt, _ = oracle.insert_trilinear(w.grid, w.images, w.poses, w.calibration(),
                                               w.spacing, w.origin)
            hit = Wt > 0
        zyx = np.argwhere(hit)
        assert len(zyx) > 0
        got_lo, got_hi = zyx.min(axis=0)[::-1], zyx.max(axis=0)[::-1] + 1
        lo, hi = _box(w, w.poses)
        assert np.all(np.asarray(lo) <= got_lo) and np.all(np.asarray(hi) >= got_hi)
        n = np.asarray(w.grid)
        if w.mode == "pnn":   # a linear frame's corners are its extremes: the box is tight
            assert np.all(got_lo - np.asarray(lo) <= 3) and np.all(np.asarray(hi) - got_hi <= 3)
        else:                 # a fan's bounding rectangle overshoots its arc a little
            assert np.all((np.asarray(hi) - np.asarray(lo)) <= 1.2 * (got_hi - got_lo) + 6)
        lo2, hi2 = _box(w, w.poses, margin=2)
        assert np.all(np.asarray(lo2) == np.maximum(np.asarray(lo) - 2, 0))
        assert np.all(np.asarray(hi2) == np.minimum(np.asarray(hi) + 2, n))
    # frames the insertion skips do not count; none left: an empty box
    bad = np.array(cases[0].poses[:1])
    bad[0, 3, 3] = 2.0
    assert _box(cases[0], bad) == ((0, 0, 0), (0, 0, 0))


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
    from helpers import assert_pnn_bit_exact, assert_trilinear_close, oracle_run
    for s, w in ((s1, w1), (s2, w2), (s3, w3)):
        torch.cuda.synchronize()
        o = oracle_run(w)
        # the region-refreshed image and the streamed accumulators, against
        # the oracle of every frame of the scan
        g = dict(band=w.band, proj=s.out.cpu().numpy(),
                 pcnt=s.cnt.cpu().numpy().view(np.uint16))
        acc = s.vol.read(usvol.READ_ACCUM).cpu().numpy()
        s.vol.fill()
        g["val"] = s.vol.read(usvol.READ_VALUES).cpu().numpy()
        g["has"] = s.vol.read(usvol.READ_MASK).cpu().numpy()
        if w.mode == "pnn":
            acc = acc.view(np.uint64)
            g["sum"] = acc & np.uint64(0xFFFFFFFF)
            g["cnt"] = (acc >> np.uint64(32)).astype(np.uint32)
            assert_pnn_bit_exact(g, o)
        else:
            g["S"] = acc[..., 0].astype(np.float64)
            g["W"] = acc[..., 1].astype(np.float64)
            assert_trilinear_close(g, o)
        # and it equals a full refresh of the streamed volume
        full, fcnt = s.vol.project(*w.band)
        torch.cuda.synchronize()
        assert torch.equal(s.out, full) and torch.equal(s.cnt, fcnt)
