"""The bounds-checked build (compiled with -DUSV_CHECKED: every kernel write
and every shared-memory accumulation tests its index, and an index outside
its buffer is skipped and raises USV_STATUS_OOB, which usvol.status()
turns into an error): the small-grid GPU parity tests run once more against
it, in a child process with USV_CHECKED=1 -- random geometries and tile
shapes of both insertions, hand-built fills, the volume life cycles and the
multi-volume insertion.  They must pass, with their oracle comparisons, and
no write may stray."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_small_grid_suite_passes_on_the_checked_build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_00058_gb300 import build
    build.build(checked=True)
    files = ["tests/test_gpu_fuzz.py", "tests/test_gpu_tiles.py", "tests/test_gpu_pnn.py",
             "tests/test_gpu_cycles.py", "tests/test_gpu_multi.py", "tests/test_golden.py"]
    env = dict(os.environ, USV_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-q", "-m", "gpu and not slow",
                        "-p", "no:cacheprovider", "-x"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
