"""Volume life cycles against the oracle, bit for bit, on both plane loaders
of the fill (tensor copies for even nx, 8-byte copies for odd nx): probe
sweeps that move through the volume from one fill-and-clear cycle to the
next (the two accumulator sets swap every cycle, each must come back
zeroed), incremental inserts between fills, a reset between inserts, and
several volumes filled by one multi-job insertion then cleared."""
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


def _sweep(grid, y0_mm, seed, n=20):
    from paper_2412_00058_gb300 import synth
    return synth.tiny_pnn(seed=seed, n=n, H=64, W=80, px=0.2, grid=grid, tilt_deg=8.0,
                          sweep_mm=6.0, y0_mm=y0_mm, band=(10, 40))


def _dev(w):
    import torch
    from paper_2412_00058_gb300 import usvol
    return (torch.from_numpy(np.ascontiguousarray(w.images)).cuda(),
            torch.from_numpy(np.ascontiguousarray(w.poses)).cuda(), usvol.calibration_of(w))


def _check(vol, w, out, cnt, o=None):
    from paper_2412_00058_gb300 import usvol
    o = oracle_run(w) if o is None else o
    assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), o["val"])
    assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), o["has"])
    assert np.array_equal(out.cpu().numpy(), o["proj"])
    assert np.array_equal(cnt.cpu().numpy().view(np.uint16), o["pcnt"])


@pytest.mark.parametrize("nx", [96, 95])
def test_moving_sweeps_over_fill_and_clear_cycles(nx):
    """Each cycle inserts a sweep elsewhere in y (the third overlaps the
    second), then fills with in-pass clearing: every cycle equals the oracle
    of its own frames, and the accumulators are zero after each."""
    from paper_2412_00058_gb300 import usvol
    grid = (nx, 200, 64)
    vol = usvol.Volume(grid, (0.3,) * 3, (0.0, 0.0, 0.0), "pnn", spare=True)
    vol.reset()
    for k, y0 in enumerate([5.0, 20.0, 23.0, 40.0, 5.0]):
        w = _sweep(grid, y0, seed=50 + k)
        vol.insert(*_dev(w))
        vol.fill_and_clear()
        out, cnt = vol.project(*w.band)
        _check(vol, w, out, cnt)
        assert not vol.read(usvol.READ_ACCUM).cpu().numpy().any()
    assert vol.status() == 0


@pytest.mark.parametrize("nx", [96, 95])
def test_incremental_inserts_between_fills_and_reset(nx):
    """Insert A, fill; insert B, fill (the union); reset; insert C, fill:
    only C's data remains."""
    from paper_2412_00058_gb300 import usvol
    grid = (nx, 200, 64)
    a, b, c = (_sweep(grid, y0, seed=70 + k) for k, y0 in enumerate([8.0, 30.0, 45.0]))
    vol = usvol.Volume(grid, (0.3,) * 3, (0.0, 0.0, 0.0), "pnn")
    vol.reset()
    vol.insert(*_dev(a))
    vol.fill()
    out, cnt = vol.project(*a.band)
    _check(vol, a, out, cnt)
    vol.insert(*_dev(b))
    vol.fill()
    out, cnt = vol.project(*a.band)
    ab = oracle_run(a, images=np.concatenate([a.images, b.images]),
                    poses=np.concatenate([a.poses, b.poses]))
    _check(vol, a, out, cnt, ab)
    vol.reset()
    vol.insert(*_dev(c))
    vol.fill()
    out, cnt = vol.project(*c.band)
    _check(vol, c, out, cnt)


def test_multi_volume_insert_then_fill_and_clear():
    """Two volumes filled by one multi-job insertion, then cleared and
    refilled with each other's sweep."""
    from paper_2412_00058_gb300 import usvol
    grid = (96, 200, 64)
    ws = [_sweep(grid, 10.0, seed=90), _sweep(grid, 35.0, seed=91)]
    vols = [usvol.Volume(grid, (0.3,) * 3, (0.0, 0.0, 0.0), "pnn", spare=True) for _ in ws]
    for v in vols:
        v.reset()
    for rnd in range(2):
        ws_r = ws if rnd == 0 else ws[::-1]
        usvol.insert_frames_multi([(v, *_dev(w)) for v, w in zip(vols, ws_r)])
        for v, w in zip(vols, ws_r):
            v.fill_and_clear()
            out, cnt = v.project(*w.band)
            _check(v, w, out, cnt)
            assert not v.read(usvol.READ_ACCUM).cpu().numpy().any()
