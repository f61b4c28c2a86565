"""bench.py prints one JSON line with the keys its consumers read: the CPU
reference arm (the oracle on all host cores, the whole sweep every step, or
a measured piece of it when K + W sweeps would pass the time budget; here
on a 600-frame sweep) on the CPU, and a short GPU run on a 600-frame
piece of the sweep on the GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e"}


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--frames", "600")
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "frames/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    assert 1 <= cb["cores"] <= len(os.sched_getaffinity(0))
    assert abs(d["ms_per_step"] - 600 / d["value"] * 1e3) < 1e-6 * d["ms_per_step"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert cb["frames_per_step"] == 600


def test_reference_arm_bounds_long_runs_by_a_measured_piece():
    """When K + W whole sweeps would pass the budget, a step is a piece of the
    sweep, timed as it is: ms_per_step is the piece's own time."""
    d = run_bench("--impl", "reference", "--steps", "3", "--warmup", "1", "--frames", "600",
                  "--ref-budget-s", "0.05")
    cb = d["cpu_baseline"]
    m = cb["frames_per_step"]
    assert 1 <= m < 600 and "measured, not scaled" in cb["sample"]
    assert d["steps"] == 3 and d["value"] > 0
    assert abs(d["ms_per_step"] - m / d["value"] * 1e3) < 1e-6 * d["ms_per_step"]


def test_reference_piece_slab_holds_every_pixel_of_its_frames():
    """The y-slab of a piece receives exactly what the full volume receives
    from the same frames."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    w = bench.sweep_workload(300)
    f0, m, grid, origin = bench.oracle_piece(w, 100, 60)
    fr = slice(f0, f0 + m)
    s_full, c_full, _ = oracle.insert_pnn(w.grid, w.images[fr], w.poses[fr], w.calib, w.sx,
                                          w.sy, w.spacing, w.origin)
    s, c, _ = oracle.insert_pnn(grid, w.images[fr], w.poses[fr], w.calib, w.sx, w.sy,
                                w.spacing, origin)
    y0 = int(round((origin[1] - w.origin[1]) / w.spacing[1]))
    assert grid[1] < w.grid[1] and int(c.sum()) == int(c_full.sum()) > 0
    assert np.array_equal(c, c_full[:, y0:y0 + grid[1], :])
    assert np.array_equal(s, s_full[:, y0:y0 + grid[1], :])


@pytest.mark.gpu
def test_gpu_arm_line():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    d = run_bench("--frames", "600", "--steps", "4", "--warmup", "3", "--e2e-steps", "2",
                  "--stream-seconds", "0", "--no-variants", "--no-cpu-baseline")
    assert BASE_KEYS <= set(d)
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 4 and d["warmup"] == 3
    assert d["gpu_launches"] == 4 * 4
    rl = d["roofline"]
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and 0 < rl["frac"] < 2
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 600 * 640 * 480 + 600 * 128
    assert e["d2h_bytes_per_step"] > 0
    assert e["host_link"]["h2d_gbs"] > 0 and 0 < e["host_link"]["frac"] < 1.5
    hl = e["host_link"]
    assert hl["h2d_gbs"] == max(hl["h2d_gbs_before"], hl["h2d_gbs_after"])
    assert len(e["runs_ms_per_step"]) == 3
    assert e["ms_per_step"] == sorted(e["runs_ms_per_step"])[1]
    pr = d["pipeline_roofline"]
    assert pr["clear_bytes_per_step"] > 0 and 0 < pr["frac"] < 2
    assert set(d["stage_ms"]) == {"insert", "fill", "project", "gaps"}
    assert d["cuda_graph"]["ms_per_step"] > 0 and d["autotune"]["tile"]
    clocks = d["clocks"]
    assert clocks is None or "sm_mhz" in clocks


def test_kernel_record_is_used_only_for_its_own_source(tmp_path):
    """roofline.traffic and the issue roofline come from the committed ncu
    record of the insertion kernel only while the kernel source still has the
    record's sha256; a record of another source gives nothing."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    kernel = tmp_path / "k.cu"
    kernel.write_text("// a kernel\n")
    sha = hashlib.sha256(kernel.read_bytes()).hexdigest()
    rec = tmp_path / "rec.txt"
    body = ("# comment = ignored\nkernel = k\nsource_sha256 = {}\n"
            "dram_bytes_read = 1.5e9\ndram_bytes_write = 0.5e9\nwarp_inst_per_pixel = 0.5\n")
    rec.write_text(body.format(sha))
    kv = bench.insert_record(str(kernel), str(rec))
    assert float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"]) == 2.0e9
    assert kv["warp_inst_per_pixel"] == "0.5" and "comment" not in kv
    rec.write_text(body.format("0" * 64))
    assert bench.insert_record(str(kernel), str(rec)) == {}
    kernel.write_text("// a kernel, changed\n")
    rec.write_text(body.format(sha))
    assert bench.insert_record(str(kernel), str(rec)) == {}
