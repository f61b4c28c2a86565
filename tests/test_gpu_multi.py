"""Several (volume, frames) jobs in one launch pair (usv_insert_frames_multi):
every volume ends bit-identical to inserting its own job alone, and to the
CPU oracle."""
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


def _workloads():
    from paper_2412_00058_gb300 import synth
    return [
        synth.tiny_pnn(n=64),
        synth.whole_spine(n=47, grid=(270, 90, 200), y_start_mm=3.0, y_span_mm=20.0),
        synth.tiny_pnn(seed=5, n=9, H=37, W=100, px=0.21, grid=(48, 40, 44), tilt_deg=15.0,
                       sweep_mm=5.0, y0_mm=3.0, band=(3, 30)),   # per-byte loads
        synth.tiny_pnn(seed=6, n=1, H=48, W=64, grid=(40, 40, 40), sweep_mm=1.0, y0_mm=4.0),
        synth.tiny_pnn(seed=7, n=0, H=48, W=64, grid=(40, 40, 40)),
    ]


def _accum(vol):
    from paper_2412_00058_gb300 import usvol
    return vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64)


def _on_device(w):
    import torch
    from paper_2412_00058_gb300 import usvol
    return (torch.from_numpy(np.ascontiguousarray(w.images)).cuda(),
            torch.from_numpy(np.ascontiguousarray(w.poses.reshape(-1, 16))).cuda(),
            usvol.calibration_of(w))


def test_multi_insert_equals_separate_inserts_and_oracle():
    from paper_2412_00058_gb300 import usvol
    ws = _workloads()
    dev = [_on_device(w) for w in ws]
    multi = [usvol.Volume(w.grid, w.spacing, w.origin, "pnn") for w in ws]
    alone = [usvol.Volume(w.grid, w.spacing, w.origin, "pnn") for w in ws]
    multi[1].set_tile(640, 480, (128, 32, 4))   # a set shape applies to its job
    for v in multi + alone:
        v.reset()
    usvol.insert_frames_multi([(v, i, p, c) for v, (i, p, c) in zip(multi, dev)])
    usvol.insert_frames_multi([(v, i, p, c) for v, (i, p, c) in zip(multi, dev)])  # twice
    for v, (i, p, c) in zip(alone, dev):
        if i.shape[0]:
            v.insert(i, p, c)
            v.insert(i, p, c)
    for w, vm, va in zip(ws, multi, alone):
        assert np.array_equal(_accum(vm), _accum(va))
        assert vm.status() == 0
    o = oracle_run(ws[1])
    acc = _accum(multi[1])
    assert np.array_equal(acc >> np.uint64(32), 2 * o["cnt"].astype(np.uint64))
    assert np.array_equal(acc & np.uint64(0xFFFFFFFF), 2 * o["sum"].astype(np.uint64))


def test_multi_insert_many_small_jobs():
    """32 jobs (the most a launch takes) of 1-5 frames each."""
    from paper_2412_00058_gb300 import synth, usvol
    rng = np.random.default_rng(3)
    jobs, alone = [], []
    for k in range(32):
        w = synth.tiny_pnn(seed=100 + k, n=int(rng.integers(1, 6)), H=40, W=48,
                           grid=(48, 48, 48), sweep_mm=3.0, y0_mm=2.0 + 0.1 * k)
        i, p, c = _on_device(w)
        vm = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
        va = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
        vm.reset()
        va.reset()
        va.insert(i, p, c)
        jobs.append((vm, i, p, c))
        alone.append(va)
    usvol.insert_frames_multi(jobs)
    for (vm, _, _, _), va in zip(jobs, alone):
        assert np.array_equal(_accum(vm), _accum(va))


def test_multi_insert_errors():
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    w = synth.tiny_pnn(n=3, H=32, W=32, grid=(40, 40, 40))
    i, p, c = _on_device(w)
    a = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    b = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
    t = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear")

    def code(jobs):
        with pytest.raises(usvol.UsvError) as e:
            usvol.insert_frames_multi(jobs)
        return e.value.code

    assert code([(a, i, p, c), (a, i, p, c)]) == usvol.ERR_ARG
    assert code([(a, i, p, c), (t, i, p, c)]) == usvol.ERR_UNSUPPORTED
    big = torch.zeros((4097, 2, 8), dtype=torch.uint8, device="cuda")
    bigp = p[:1].repeat(4097, 1).contiguous()
    assert code([(b, big, bigp, c)]) == usvol.ERR_RANGE
    vols = [usvol.Volume(w.grid, w.spacing, w.origin, "pnn") for _ in range(33)]
    assert code([(v, i, p, c) for v in vols]) == usvol.ERR_RANGE
    usvol.insert_frames_multi([])  # nothing to do


def test_volumes_driven_from_several_host_threads():
    """Four host threads, each with its own volume and stream (insert, fill
    with clearing, projection): each equals the same work done alone."""
    import threading
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    ws = [synth.tiny_pnn(seed=40 + k, n=20, H=64, W=64, grid=(64, 64, 64), sweep_mm=5.0,
                         band=(20, 40))
          for k in range(4)]
    dev = [_on_device(w) for w in ws]
    vols = [usvol.Volume(w.grid, w.spacing, w.origin, "pnn", spare=True) for w in ws]
    outs = [None] * 4
    errors = []

    def work(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                v = vols[k]
                v.reset(st)
                for _ in range(3):
                    v.insert(*dev[k], stream=st)
                    v.fill_and_clear(st)
                outs[k] = v.project(*ws[k].band, stream=st)
            st.synchronize()
        except Exception as e:  # reported in the main thread
            errors.append(e)

    th = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    for k, w in enumerate(ws):
        ref = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
        ref.reset()
        ref.insert(*dev[k])
        ref.fill()
        out, cnt = ref.project(*w.band)
        assert torch.equal(outs[k][0], out) and torch.equal(outs[k][1], cnt)


def test_multi_insert_with_tissue_cut_rows():
    """Per-frame first rows (tissue segmentation) in a multi-job insertion
    equal usv_insert_frames_cut of each job."""
    import torch
    from paper_2412_00058_gb300 import synth, usvol
    ws = [synth.whole_spine(n=30, grid=(270, 80, 200), y_start_mm=3.0, y_span_mm=10.0),
          synth.tiny_pnn(n=20)]
    rng = np.random.default_rng(9)
    jobs, alone = [], []
    for w in ws:
        i, p, c = _on_device(w)
        rows = torch.from_numpy(rng.integers(-5, w.H + 5, w.n).astype(np.int32)).cuda()
        vm = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
        va = usvol.Volume(w.grid, w.spacing, w.origin, "pnn")
        vm.reset()
        va.reset()
        usvol.insert_frames_cut(va.handle, i.data_ptr(), w.n, w.H, w.W, usvol.U8, p.data_ptr(),
                                c, rows.data_ptr())
        jobs.append((vm, i, p, c, rows))
        alone.append(va)
    usvol.insert_frames_multi(jobs)
    for (vm, *_), va in zip(jobs, alone):
        assert np.array_equal(_accum(vm), _accum(va))
        assert _accum(vm).any()
