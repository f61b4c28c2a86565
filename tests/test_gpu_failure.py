"""Device-side failure path without a GPU fault: the fill kernel's only wait
(for each plane's tensor copy) is bounded by about one second.  A test hook
withholds one plane's copy, so that wait runs out: the kernel reports
USV_STATUS_TIMEOUT through the status word, returns, and the volume and the
CUDA context stay usable (the next fill equals the oracle)."""
import time

import numpy as np
import pytest

from helpers import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build_library()


def test_bounded_wait_runs_out_and_the_volume_stays_usable():
    import torch
    import oracle
    from paper_2412_00058_gb300 import usvol
    grid = (64, 40, 20)
    nx, ny, nz = grid
    rng = np.random.default_rng(17)
    c = np.where(rng.random((nz, ny, nx)) < 0.3, rng.integers(1, 50, (nz, ny, nx)), 0)
    s = (c * rng.integers(0, 256, (nz, ny, nx))).astype(np.uint64)
    c = c.astype(np.uint32)
    packed = (c.astype(np.uint64) << np.uint64(32)) | s
    vol = usvol.Volume(grid, (0.3, 0.3, 0.3), (0, 0, 0), "pnn")
    src = torch.from_numpy(packed.view(np.int64)).cuda()
    usvol.volume_write_accum(vol.handle, src.data_ptr())
    assert vol.status() == 0

    t0 = time.perf_counter()
    usvol.fill_with_withheld_copy(vol.handle, 5)
    st = vol.status()                      # waits for the stream
    elapsed = time.perf_counter() - t0
    assert st & usvol.STATUS_TIMEOUT
    assert 0.5 < elapsed < 30.0            # the wait gave up after about a second
    assert vol.status() == 0               # read and cleared
    assert np.array_equal(vol.read(usvol.READ_ACCUM).cpu().numpy().view(np.uint64), packed)

    vol.fill()                             # the context and the volume still work
    ov, oh = oracle.fill_pnn(s, c)
    assert np.array_equal(vol.read(usvol.READ_VALUES).cpu().numpy(), ov)
    assert np.array_equal(vol.read(usvol.READ_MASK).cpu().numpy(), oh)
    assert vol.status() == 0


def test_timeout_hook_arguments():
    from paper_2412_00058_gb300 import usvol
    vol = usvol.Volume((64, 40, 20), (0.3,) * 3, (0, 0, 0), "pnn")
    for plane in (-1, 20):
        with pytest.raises(usvol.UsvError) as e:
            usvol.fill_with_withheld_copy(vol.handle, plane)
        assert e.value.code == usvol.ERR_ARG
    odd = usvol.Volume((63, 40, 20), (0.3,) * 3, (0, 0, 0), "pnn")
    with pytest.raises(usvol.UsvError) as e:
        usvol.fill_with_withheld_copy(odd.handle, 3)
    assert e.value.code == usvol.ERR_UNSUPPORTED
