#!/usr/bin/env python
"""Whole-spine sweep benchmark for the GB300 free-hand ultrasound path.

One step = one pass of the whole path over one synthetic whole-spine sweep
(3600 frames of 480x640 uint8 = 2 min at 30 fps, 550 mm along the spine):
insert all frames into the empty 270x1840x200 volume (pixel nearest
neighbour), normalise + 3x3x3 hole fill, project the 35-45 mm depth band.
The fill also clears the accumulators for the next sweep (the volume has a
spare accumulator set), so every step starts from an empty volume without a
separate reset pass.  Inputs are resident in HBM when the timed region starts
(they are larger than L2, so no flush is needed between steps).

Prints one JSON line (rank 0):
  value      frames/s of the whole job (all ranks), CUDA-event timed
  e2e        the same metric through the public API from pinned HOST buffers,
             frames streamed host->device in 300-frame batches overlapped
             with insertion, poses passed from host memory, projection read
             back every step; with the host link measured in the same run
  roofline   the dominant kernel (insertion): algorithmic bytes / its event-
             timed launch duration vs the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle on the whole sweep, on all host cores (and on
             one thread)
  clocks     nvidia-smi SM clocks / throttle reasons sampled while timing

--impl reference times the CPU oracle (the only reference: the paper
publishes no code) on the same metric: the whole sweep every step, on all
host cores.  Multi-GPU: replicas only -- every
rank reconstructs its own sweep with no collective in the data path; the
barrier and a MAX all-reduce of the elapsed time bracket the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("frames/s & voxel-updates/s (full-spine sweep) vs HBM roofline; "
          "p99 frame-to-render ms")
WORKLOAD = ("whole-spine linear-probe sweep: 3600 frames 480x640 uint8, 550 mm along y, "
            "+-20 mm sway, +-10 deg tilt; volume 270x1840x200 @ 0.3 mm; PNN insert + 3x3x3 "
            "fill + depth band [117,150)")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="usvol", choices=["usvol", "reference"])
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--ref-budget-s", type=float, default=180.0,
                   help="--impl reference: seconds of oracle work the K + W steps may take")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--variants-only", action="store_true",
                   help="run only the variant rows (for profiling them)")
    p.add_argument("--variant-frames", type=int, default=0,
                   help="convex sweep variant: only this many frames, into the y-slab they "
                        "cover (a small case for profiling)")
    p.add_argument("--no-graph", action="store_true",
                   help="skip the CUDA-graph replay of the step")
    p.add_argument("--no-tune", action="store_true",
                   help="keep the default insertion tile shape (skip the autotuner)")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the trilinear convex sweep and pose-gradient timings")
    p.add_argument("--stream-seconds", type=float, default=4.0,
                   help="seconds of the four-session streaming run (0: skip)")
    p.add_argument("--frames", type=int, default=3600,
                   help="frames of the sweep (fewer = a shorter piece at the same frame "
                        "spacing; for profiling captures)")
    return p.parse_args(argv)


# ---------------------------------------------------------------- distributed

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def init_dist(backend: str):
    import torch.distributed as dist
    rank, local, world = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, local, world


def max_over_ranks(x: float, device=None) -> float:
    """MAX all-reduce of a scalar (no-op on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 100 ms, timestamped."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.perf_counter(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return None
        inside = [p for t, p in self.samples if t0 <= t <= t1]
        if not inside:  # timed region shorter than one sample period: nearest sample
            mid = 0.5 * (t0 + t1)
            inside = [min(self.samples, key=lambda s: abs(s[0] - mid))[1]]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        mx = [num(p[2]) for p in inside if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4)
                          if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


# ---------------------------------------------------------------- host placement

def gpu_local_cpus(index: int) -> set:
    """Host CPUs on the GPU's own NUMA node (from the PCI device's
    local_cpulist), intersected with this process's CPUs; empty if unknown."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist"
        with open(path) as f:
            spec = f.read().strip()
    except (OSError, ValueError, subprocess.SubprocessError):
        return set()
    cpus = set()
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus & os.sched_getaffinity(0)


# ---------------------------------------------------------------- peaks

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def insert_record(kernel_file: str = "paper_2412_00058_gb300/csrc/k_insert_pnn.cu",
                  record: str = "profiles/insert_pnn_whole_spine_traffic.txt") -> dict:
    """The committed ncu record of the insertion kernel, or {} if the kernel
    source changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, kernel_file), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        kv = {}
        with open(os.path.join(ROOT, record)) as f:
            for line in f:
                if "=" in line and not line.lstrip().startswith("#"):
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        return kv if kv.get("source_sha256") == sha else {}
    except OSError:
        return {}


def recorded_traffic() -> float | None:
    """DRAM bytes per launch of the insertion kernel (committed ncu record)."""
    kv = insert_record()
    try:
        return float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- workload

def sweep_workload(frames: int = 3600):
    from paper_2412_00058_gb300 import synth
    if frames >= 3600:
        return synth.whole_spine()
    return synth.whole_spine(n=frames, y_span_mm=550.0 * (frames - 1) / 3599.0)


# ---------------------------------------------------------------- CPU oracle

def oracle_accumulators(w, grid=None):
    """Oracle accumulators (sums, counts) of the full volume (or of `grid`),
    every page written once here, so that no timed call pays for first-touch
    page faults."""
    import numpy as np
    nx, ny, nz = grid if grid is not None else w.grid
    s = np.empty((nz, ny, nx), np.uint64)
    c = np.empty((nz, ny, nx), np.uint32)
    s.fill(0)
    c.fill(0)
    return s, c


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def oracle_sweep_seconds(w, threads: int = 1, acc=None, piece=None):
    """Time the oracle on the whole sweep: every frame inserted into the full
    volume, then fill and projection of the whole volume, on `threads` host
    threads (1: the plain single-thread loops).  piece = (f0, m, grid,
    origin) times frames [f0, f0 + m) into that y-slab of the volume
    instead (oracle_piece).  The accumulators are zeroed before the timed
    calls.  Returns (seconds, threads used)."""
    import oracle
    grid, origin, f0, m = w.grid, w.origin, 0, w.n
    if piece is not None:
        f0, m, grid, origin = piece
    s, c = acc if acc is not None else oracle_accumulators(w, grid)
    s.fill(0)
    c.fill(0)
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        oracle.insert_pnn(grid, w.images[f0:f0 + m], w.poses[f0:f0 + m], w.calib, w.sx, w.sy,
                          w.spacing, origin, sum_=s, cnt=c)
        val, has = oracle.fill_pnn(s, c)
        oracle.project_u8(val, has, *w.band)
        t = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return t, used


def oracle_piece(w, f0: int, m: int):
    """Frames [f0, f0 + m) of the sweep and the y-slab of the full grid that
    holds them: whole voxel rows from 1 mm before the frames' lowest image
    corner to 1 mm past their highest (a linear frame is flat, so its
    corners bound it).  Returns (f0, m, grid, origin)."""
    import numpy as np
    H, W = w.images.shape[1:]
    corners = np.array([[j * w.sx, 0.0, i * w.sy, 1.0]
                        for i in (0, H - 1) for j in (0, W - 1)]).T
    y = (w.poses[f0:f0 + m] @ np.asarray(w.calib) @ corners)[:, 1, :]
    sp = w.spacing[1]
    y0 = max(0, int(np.floor((y.min() - 1.0 - w.origin[1]) / sp)))
    y1 = min(w.grid[1], int(np.ceil((y.max() + 1.0 - w.origin[1]) / sp)) + 1)
    grid = (w.grid[0], y1 - y0, w.grid[2])
    origin = (w.origin[0], w.origin[1] + y0 * sp, w.origin[2])
    return f0, m, grid, origin


def measure_variants(dev, reps: int = 5, frames: int = 0, tune: bool = True):
    """Event-timed variant rows: the full convex-fan sweep with trilinear
    splatting (3000 frames 512x512 -> 400x1700x400), and one evaluation of
    the pose-refinement loss + gradient (512 FP32 frames 256x256 ->
    256x512x192)."""
    import numpy as np
    import torch
    from paper_2412_00058_gb300 import posegrad, synth, usvol
    out = {}
    stream = torch.cuda.current_stream(dev)
    if frames:  # the first `frames` frames of the sweep, into the y-slab they cover
        ny = int(660.0 * frames / 2999.0 / 0.4) + 60
        w = synth.convex_fan(n=frames, grid=(400, ny, 400), sweep_mm=660.0 * frames / 2999.0)
    else:
        w = synth.convex_fan()
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear", device=dev)
    imgs = torch.from_numpy(w.images).to(dev)
    poses = torch.from_numpy(w.poses).to(dev)
    cal = usvol.calibration_of(w)
    tri_tile = vol.tune(imgs, poses, cal, stream)[0] if tune else vol.get_tile(w.H, w.W)
    nx, ny, nz = w.grid
    img_out = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    cnt = torch.empty((ny, nx), dtype=torch.int16, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ts = []
    for r in range(reps + 1):
        ev[0].record(stream)
        vol.reset(stream)
        ev[1].record(stream)
        vol.insert(imgs, poses, cal, stream)
        ev[2].record(stream)
        vol.fill(stream)
        ev[3].record(stream)
        vol.project(*w.band, out=img_out, count=cnt, stream=stream)
        ev[4].record(stream)
        torch.cuda.synchronize(dev)
        if r:
            ts.append([ev[0].elapsed_time(ev[4])] +
                      [ev[k].elapsed_time(ev[k + 1]) for k in range(4)])
    med = [float(np.median([t[k] for t in ts])) for k in range(5)]
    step, ins = med[0], med[2]
    nvox = nx * ny * nz
    # the fill's bytes: 8 B (S, W) read + 4 B value + 1/8 B mask per voxel
    tri_fill_bytes = nvox * (8 + 4) + nz * ny * ((nx + 31) // 32) * 4
    samples = w.n * w.H * w.W
    # distinct voxels the sweep's one insertion launch touches (W > 0 after
    # the last repetition's insert) and the insert's algorithmic bytes:
    # 1 B per uint8 sample + 16 B per touched voxel (read + write of S, W)
    vol.reset(stream)
    vol.insert(imgs, poses, cal, stream)
    acc = vol.read(usvol.READ_ACCUM, stream)
    touched = int((acc[..., 1] > 0).sum().item())
    del acc
    peak, peak_kind = measured_peaks()
    tri_bytes = samples * w.images.itemsize + 16 * touched
    # the float2 vector-atomic ceiling: the library's probe, event-timed, into
    # an L2-resident 64 MB buffer and a 2 GB one
    ceil = {}
    for label, nbytes in (("l2_64MB", 64 << 20), ("hbm_2GB", 2 << 30)):
        buf = torch.zeros(nbytes // 4, dtype=torch.float32, device=dev)
        reds = 64
        nthreads = torch.cuda.get_device_properties(dev).multi_processor_count * 8 * 256
        usvol.probe_red_f2(buf.data_ptr(), nbytes, reds, stream)   # warm-up
        t_red = []
        for _ in range(3):
            ev[0].record(stream)
            usvol.probe_red_f2(buf.data_ptr(), nbytes, reds, stream)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            t_red.append(ev[0].elapsed_time(ev[1]))
        ceil[label] = nthreads * reds / (min(t_red) / 1e3)
        del buf
    out["trilinear_convex_sweep"] = {
        "workload": f"{w.n} convex frames 512x512 uint8 (60 deg, 120 mm) -> "
                    f"{w.grid[0]}x{w.grid[1]}x{w.grid[2]} @ 0.4 mm",
        "ms_per_sweep": step, "frames_per_s": w.n / step * 1e3,
        "insert_ms": ins, "samples_per_s": samples / ins * 1e3, "tile": list(tri_tile),
        "stage_ms": {"reset": med[1], "insert": med[2], "fill": med[3], "project": med[4]},
        "fill_roofline": {"bound": "hbm", "algorithmic_bytes": tri_fill_bytes,
                          "achieved": tri_fill_bytes / (med[3] / 1e3) / 1e9, "peak": peak,
                          "unit": "GB/s",
                          "frac": tri_fill_bytes / (med[3] / 1e3) / 1e9 / peak},
        "touched_voxels": touched,
        "roofline": {"bound": "hbm", "algorithmic_bytes": tri_bytes,
                     "achieved": tri_bytes / (ins / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": tri_bytes / (ins / 1e3) / 1e9 / peak, "peak_kind": peak_kind},
        "float2_atomic_ceiling_per_s": ceil,
        "what": "algorithmic bytes = 1 B per uint8 sample + 16 B per voxel the launch touches; "
                "the atomic ceilings are coalesced float2 reductions (usv_probe_red_f2) into an "
                "L2-resident and an HBM-sized buffer"}
    del vol, imgs, poses
    torch.cuda.empty_cache()
    w = synth.pose_refine()
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear", device=dev)
    prob = posegrad.PoseProblem(vol, torch.from_numpy(w.images).to(dev),
                                torch.from_numpy(w.meta["noisy_poses"]).to(dev),
                                usvol.calibration_of(w), w.band,
                                torch.zeros((w.grid[1], w.grid[0]), dtype=torch.float32,
                                            device=dev), 1e-2)
    gt = torch.from_numpy(w.poses).to(dev)
    prob.evaluate(gt)
    prob.target = prob.proj.clone()
    ts = []
    for r in range(reps + 1):
        ev[0].record(stream)
        prob.evaluate(prob.poses)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        if r:
            ts.append(ev[0].elapsed_time(ev[1]))
    out["pose_gradient"] = {
        "workload": "512 FP32 frames 256x256 -> 256x512x192 @ 0.3 mm, band [80,140)",
        "ms_per_loss_and_gradient": float(np.median(ts)),
        "loss_at_noisy_poses": float(prob.loss.item())}

    # refinement from the noisy poses toward the true poses' projection
    def errors(P):
        P = np.asarray(P).reshape(-1, 4, 4)
        T = w.poses
        t = np.abs(P[:, :3, 3] - T[:, :3, 3]).mean(axis=0)
        R = np.einsum("fij,fkj->fik", P[:, :3, :3], T[:, :3, :3])
        ang = np.degrees(np.arccos(np.clip((np.trace(R, axis1=1, axis2=2) - 1) / 2, -1, 1)))
        return {"t_mm_xyz": [float(x) for x in t], "rot_deg": float(ang.mean())}
    steps = 200
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    refined, hist = posegrad.refine(prob, steps=steps)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    out["pose_refinement"] = {
        "workload": "the same 512 frames, poses perturbed by N(0, 1 mm) and N(0, 1 deg); target: "
                    "the projection at the true poses",
        "steps": steps, "loss_before": hist[0], "loss_after": hist[-1],
        "mean_abs_error_before": errors(w.meta["noisy_poses"]),
        "mean_abs_error_after": errors(refined.cpu().numpy()),
        "ms_per_step": wall / steps * 1e3,
        "what": "per-frame normalised descent steps with backtracking (posegrad.refine); each "
                "step is one or more loss + gradient evaluations on the GPU plus host control; "
                "x (lateral) and z (depth) are observed by the depth-band projection, y (along "
                "the sweep) is not"}
    return out


def run_reference(args):
    """The oracle (the only reference: the paper publishes no code) as it
    stands, on all host cores.  A step is the whole sweep while K + W of them
    fit in --ref-budget-s; beyond that a step is the largest piece of the
    sweep (consecutive frames from its middle, with the y-slab of the volume
    they reach) that fits, timed as it is, never scaled up."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_2412_00058_gb300 import synth
    import oracle
    oracle.build()
    w = synth.whole_spine() if args.frames >= 3600 else sweep_workload(args.frames)
    acc = oracle_accumulators(w)
    cores = host_cores()
    # the first warm-up step (a calibration run when W = 0) sizes the sample
    t_full, _ = oracle_sweep_seconds(w, cores, acc)
    runs = args.steps + max(args.warmup - 1, 0)
    piece = None
    if runs * t_full > args.ref_budget_s:
        # frames per step in proportion to the budget, then once more from a
        # timed piece (the slab's fill does not shrink with the frames)
        m, t_m = w.n, t_full
        for _ in range(2):
            m = max(1, min(w.n, int(m * args.ref_budget_s / (runs * t_m))))
            piece = oracle_piece(w, (w.n - m) // 2, m)
            acc = oracle_accumulators(w, piece[2])
            t_m, _ = oracle_sweep_seconds(w, cores, acc, piece)
    for _ in range(max(args.warmup - 1, 0)):
        oracle_sweep_seconds(w, cores, acc, piece)
    times, used = [], 1
    for _ in range(args.steps):
        t, used = oracle_sweep_seconds(w, cores, acc, piece)
        times.append(t)
    total = sum(times)
    frames = w.n if piece is None else piece[1]
    value = frames * len(times) / total
    if piece is None:
        sample = (f"the whole sweep every step ({w.n} frames inserted into the full "
                  f"{w.grid[0]}x{w.grid[1]}x{w.grid[2]} volume, fill and projection of the "
                  f"whole volume)")
    else:
        f0, m, g, o = piece
        y0 = int(round((o[1] - w.origin[1]) / w.spacing[1]))
        sample = (f"frames [{f0},{f0 + m}) of the {w.n}-frame sweep every step, inserted into "
                  f"the y-slab [{y0},{y0 + g[1]}) of the {w.grid[1]}-row volume that holds "
                  f"them, fill and projection of that slab (the whole sweep, {t_full:.2f} s a "
                  f"step, would not fit {args.steps}+{args.warmup} steps in "
                  f"{args.ref_budget_s:.0f} s); measured, not scaled")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": used, "kind": "oracle",
                         "sample": sample + f"; accumulators zeroed before each step outside "
                                            f"its timing; {used} threads",
                         "frames_per_step": frames},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def run_gpu(args):
    import numpy as np
    import torch

    rank, local, world = init_dist("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2412_00058_gb300 import build, synth, usvol
    if rank == 0 or world == 1:
        build.build()
    barrier(dev)
    usvol.lib()
    if args.variants_only:
        if rank == 0:
            print(json.dumps({"variants": measure_variants(dev, frames=args.variant_frames,
                                                           tune=not args.no_tune)}), flush=True)
        return 0

    w = sweep_workload(args.frames)
    nx, ny, nz = w.grid
    lo, hi = w.band
    # a spare accumulator set lets the fill clear the accumulators for the
    # next sweep in the same pass (no separate reset pass over 795 MB)
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "pnn", device=dev, spare=True)
    imgs = torch.from_numpy(w.images).to(dev)
    poses = torch.from_numpy(w.poses).to(dev)
    cal = usvol.calibration_of(w)
    out = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    cnt = torch.empty((ny, nx), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    launches_per_step = 4  # insert: set-up + insert; fill (+ clear); project

    def step(ev=None):
        # starts on zero accumulators: the previous step's fill cleared them
        if ev is not None:
            ev[0].record(stream)
        vol.insert(imgs, poses, cal, stream)
        if ev is not None:
            ev[1].record(stream)
        vol.fill_and_clear(stream)
        if ev is not None:
            ev[2].record(stream)
        vol.project(lo, hi, out=out, count=cnt, stream=stream)
        if ev is not None:
            ev[3].record(stream)

    # insertion tile shape: the project's autotuner on this sweep's frames
    tune = None
    if not args.no_tune:
        t_t0 = time.perf_counter()
        tile, tile_ms = vol.tune(imgs, poses, cal, stream)
        tune = {"tile": list(tile), "default": [128, 64, 12],
                "insert_ms_tuning_frames": tile_ms, "tuning_frames": min(w.n, 4096), "candidates": 50,
                "seconds": time.perf_counter() - t_t0}
    vol.reset(stream)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    st = vol.status(stream)
    if st != 0:
        raise RuntimeError(f"device status {st:#x} after warm-up")
    # distinct voxels touched by one sweep (one insert launch) and pixel hits,
    # from one untimed insert; its fill clears the accumulators again
    vol.insert(imgs, poses, cal, stream)
    acc = vol.read(usvol.READ_ACCUM, stream)
    counts = (acc >> 32)
    touched = int((counts > 0).sum().item())
    hits = int(counts.sum().item())
    del acc, counts
    vol.fill_and_clear(stream)
    torch.cuda.synchronize(dev)

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    e_start = torch.cuda.Event(enable_timing=True)
    e_stop = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index).start() if rank == 0 else None
    time.sleep(0.25 if sampler else 0.0)
    barrier(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e_start.record(stream)
    for k in range(K):
        step(evs[k])
    e_stop.record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    barrier(dev)
    if sampler:
        sampler.stop()
    local_ms = e_start.elapsed_time(e_stop)
    total_ms = max_over_ranks(local_ms, dev)
    ms_per_step = total_ms / K
    ins_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    fill_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    proj_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    frames = w.n * world * K
    value = frames / (total_ms / 1e3)
    vupd = hits * world * K / (total_ms / 1e3)

    # ---- the same step replayed from a captured CUDA graph (two steps per
    # graph: the accumulator sets swap at every step)
    graph = None
    if not args.no_graph:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for _ in range(2):
                vol.insert(imgs, poses, cal)
                vol.fill_and_clear()
                vol.project(lo, hi, out=out, count=cnt)
        torch.cuda.synchronize(dev)
        for _ in range(2):
            g.replay()
        reps = max(1, K // 2)
        ge0, ge1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ge0.record(stream)
        for _ in range(reps):
            g.replay()
        ge1.record(stream)
        torch.cuda.synchronize(dev)
        graph = {"ms_per_step": ge0.elapsed_time(ge1) / (2 * reps), "steps_per_graph": 2,
                 "replays": reps}
        del g

    # ---- the same sweep inserted as it is acquired: 120 calls of 30 frames
    # (one second at 30 fps each), then fill and projection
    b30 = None
    if not args.no_graph:
        reps30 = 20
        torch.cuda.synchronize(dev)
        be0, be1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        be0.record(stream)
        for _ in range(reps30):
            for b0 in range(0, w.n, 30):
                vol.insert(imgs[b0:b0 + 30], poses[b0:b0 + 30], cal, stream)
            vol.fill_and_clear(stream)
            vol.project(lo, hi, out=out, count=cnt, stream=stream)
        be1.record(stream)
        torch.cuda.synchronize(dev)
        ms30 = be0.elapsed_time(be1) / reps30
        b30 = {"ms_per_sweep": ms30, "frames_per_s": w.n / ms30 * 1e3,
               "inserts_per_sweep": (w.n + 29) // 30}

    # ---- roofline of the dominant kernel (insertion)
    peak, peak_kind = measured_peaks()
    nvox = nx * ny * nz
    frame_bytes = w.images.nbytes
    ins_bytes = frame_bytes + 16 * touched
    achieved = ins_bytes / (ins_ms / 1e3) / 1e9
    fill_bytes = nvox * (8 + 1) + nz * ny * ((nx + 31) // 32) * 4
    proj_bytes = (hi - lo) * ny * (nx + ((nx + 31) // 32) * 4 / 1) + ny * nx * 6
    # zeros for the next sweep, written by the fill: work of every step, but
    # not bytes the method moves, so not counted in the fractions
    clear_bytes = nvox * 8
    step_bytes = ins_bytes + fill_bytes + proj_bytes

    # ---- end to end through the public API from pinned host memory: every
    # step copies its sweep host->device (12 batches of 300 frames on a copy
    # stream, each batch inserted as soon as it has landed, its poses passed
    # from host memory: the library stages them) and reads its projection
    # back.  Two device frame buffers let the next sweep's copies start while
    # this sweep is still being filled and projected; the host waits once,
    # after the last step.  The pinned buffers are placed on the GPU's own
    # NUMA node, and the host link is measured in the same run (one 1.1 GB
    # pinned host->device copy, best of 3).
    e2e = None
    if args.e2e_steps > 0:
        local = gpu_local_cpus(dev.index)
        prev_aff = os.sched_getaffinity(0)
        if local:
            os.sched_setaffinity(0, local)   # first touch of the pinned pages: local node
        try:
            h_imgs = torch.from_numpy(w.images).pin_memory()
            h_poses = torch.from_numpy(w.poses).pin_memory()
            h_out = [torch.empty((ny, nx), dtype=torch.float32).pin_memory() for _ in range(2)]
            h_cnt = [torch.empty((ny, nx), dtype=torch.int16).pin_memory() for _ in range(2)]
        finally:
            os.sched_setaffinity(0, prev_aff)
        d_imgs = [imgs, torch.empty_like(imgs)]
        copy_stream = torch.cuda.Stream(dev)
        batch = 300
        bounds = [(b, min(w.n, b + batch)) for b in range(0, w.n, batch)]
        freed = [None, None]  # per buffer: the inserts that last read it

        # the host link: the same bytes in one pinned host->device copy, best
        # of 3, measured before and after the end-to-end runs (the host's
        # memory is shared with other GPUs' jobs, so the rate can drift)
        le0, le1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def link_rate():
            link = []
            with torch.cuda.stream(copy_stream):
                for _ in range(3):
                    le0.record(copy_stream)
                    d_imgs[1].copy_(h_imgs, non_blocking=True)
                    le1.record(copy_stream)
                    le1.synchronize()
                    link.append(h_imgs.numel() / (le0.elapsed_time(le1) / 1e3) / 1e9)
            return max(link)
        link_before = link_rate()

        def e2e_steps(k_steps):
            for k in range(k_steps):
                buf = k % 2
                landed = []
                with torch.cuda.stream(copy_stream):
                    if freed[buf] is not None:
                        copy_stream.wait_event(freed[buf])
                    for b0, b1 in bounds:
                        d_imgs[buf][b0:b1].copy_(h_imgs[b0:b1], non_blocking=True)
                        e = torch.cuda.Event()
                        e.record(copy_stream)
                        landed.append(e)
                for (b0, b1), e in zip(bounds, landed):
                    stream.wait_event(e)
                    vol.insert(d_imgs[buf][b0:b1], h_poses[b0:b1], cal, stream)
                freed[buf] = torch.cuda.Event()
                freed[buf].record(stream)
                vol.fill_and_clear(stream)
                vol.project(lo, hi, out=out, count=cnt, stream=stream)
                h_out[buf].copy_(out, non_blocking=True)
                h_cnt[buf].copy_(cnt, non_blocking=True)
            stream.synchronize()
            copy_stream.synchronize()
            return (k_steps - 1) % 2

        e2e_steps(1)
        # three timed runs of K steps each; the median run is the value
        runs = []
        for _ in range(3):
            barrier(dev)
            t_e0 = time.perf_counter()
            last = e2e_steps(args.e2e_steps)
            runs.append(max_over_ranks(time.perf_counter() - t_e0, dev))
            assert np.array_equal(h_out[last].numpy(), out.cpu().numpy())
        t_e = sorted(runs)[1]
        link_after = link_rate()
        link_gbs = max(link_before, link_after)
        frames_gbs = w.images.nbytes * args.e2e_steps / t_e / 1e9
        e2e = {"value": w.n * world * args.e2e_steps / t_e, "unit": "frames/s",
               "h2d_bytes_per_step": int(w.images.nbytes + w.poses.nbytes),
               "d2h_bytes_per_step": int(h_out[0].numel() * 4 + h_cnt[0].numel() * 2),
               "ms_per_step": t_e / args.e2e_steps * 1e3,
               "runs_ms_per_step": [t / args.e2e_steps * 1e3 for t in runs],
               "host_link": {"h2d_gbs": link_gbs, "h2d_gbs_before": link_before,
                             "h2d_gbs_after": link_after, "frames_gbs": frames_gbs,
                             "frac": frames_gbs / link_gbs,
                             "pinned_on_cpus": f"{len(local)} GPU-local cpus" if local
                             else "default placement (GPU-local cpus not found)",
                             "what": "one 1.1 GB pinned host->device copy of the same frames, "
                                     "best of 3, measured before and after the three "
                                     "end-to-end runs in this run"},
               "pipeline": f"{len(bounds)} batches of {batch} frames, H2D on a copy stream "
                           "overlapped with insertion, host poses staged by the library; two "
                           "device frame buffers, so the next sweep's copies overlap this "
                           "sweep's fill and projection"}

    # ---- streaming: four concurrent sessions, frame-to-render latency
    streaming = None
    if args.stream_seconds > 0:
        from paper_2412_00058_gb300 import stream as ustream
        sessions = synth.streaming_sessions(args.stream_seconds)

        def serve(batched, realtime):
            sched = ustream.Scheduler(dev)
            for i, (name, sw, fps) in enumerate(sessions):
                sched.admit(name, sw, fps, seed=i)
            out = ustream.summary(sched.run(args.stream_seconds, batched=batched,
                                            realtime=realtime))
            out["wall_s"] = sched.wall_s
            if batched:
                out["dispatches"] = sched.dispatches
            del sched
            torch.cuda.synchronize(dev)
            torch.cuda.empty_cache()
            return out

        streaming = serve(batched=False, realtime=True)
        streaming["seconds"] = args.stream_seconds
        streaming["what"] = ("per-frame latency from burst arrival on the host to its "
                             "region-refreshed projection completing on the device; bursts of "
                             "1-32 frames at 30/60/120/30 fps into 128^3, 256x1024x200, "
                             "270x1840x200 (PNN) and 400x1700x400 (trilinear) volumes; "
                             "one CUDA stream per session")
        bat = serve(batched=True, realtime=True)
        streaming["batched"] = {k: bat[k] for k in ("p50_ms", "p99_ms", "max_ms", "bursts",
                                                      "dispatches")}
        streaming["batched"]["what"] = ("one engine stream; each dispatch inserts every "
                                        "session's waiting burst with one multi-volume "
                                        "insertion (persistent kernel), then refreshes regions")
        rs, rb = serve(batched=False, realtime=False), serve(batched=True, realtime=False)
        streaming["replay_frames_per_s"] = {
            "per_session_streams": rs["frames"] / rs["wall_s"],
            "batched": rb["frames"] / rb["wall_s"], "batched_dispatches": rb["dispatches"],
            "what": "all bursts of the same sessions available at once, served as fast as "
                    "the GPU takes them (host wall clock, includes host->device copies)"}

    # ---- variant rows: trilinear convex sweep, pose gradient (one GPU)
    variants = None
    if not args.no_variants and world == 1:
        variants = measure_variants(dev, frames=args.variant_frames, tune=not args.no_tune)

    # ---- CPU oracle (rank 0, one GPU only): the whole sweep on one thread
    # and on every host core, each run twice (about 20 s of CPU work)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        acc = oracle_accumulators(w)
        one = [oracle_sweep_seconds(w, 1, acc)[0] for _ in range(2)]
        multi = [oracle_sweep_seconds(w, host_cores(), acc) for _ in range(2)]
        used = multi[0][1]
        t_all = sum(t for t, _ in multi) / len(multi)
        del acc
        cpu = {"value": w.n / t_all, "unit": "frames/s", "cores": used, "kind": "oracle",
               "sample": f"the whole sweep ({w.n} frames into the full volume, fill and "
                         f"projection of the whole volume) on {used} host threads, run twice, "
                         f"mean",
               "single_thread": {"value": w.n / (sum(one) / len(one)), "unit": "frames/s",
                                 "cores": 1, "sample": "the same sweep on one thread, twice"}}

    clocks = sampler.summary(t0, t1) if sampler else None
    # the insertion kernel against the instruction-issue roofline: 4 warp
    # schedulers per SM, one warp instruction each per clock, at the SM clock
    # sampled while timing (the maximum clock if there was no sample)
    issue = None
    kv = insert_record()
    if "warp_inst_per_pixel" in kv:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
        if mhz:
            ipp = float(kv["warp_inst_per_pixel"])
            got = ipp * w.n * w.H * w.W / (ins_ms / 1e3)
            top = sms * 4 * mhz * 1e6
            issue = {"bound": "issue", "achieved": got, "peak": top, "unit": "warp-instr/s",
                     "frac": got / top, "warp_inst_per_pixel": ipp,
                     "source": "warp instructions per pixel from the committed ncu record of "
                               "the same kernel source; peak = SMs x 4 schedulers x SM clock"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (1.1 GB frames, 795 MB accumulators)"},
            "voxel_updates_per_s": vupd,
            "stage_ms": {"insert": ins_ms, "fill": fill_ms, "project": proj_ms,
                         "gaps": ms_per_step - ins_ms - fill_ms - proj_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic() if args.frames >= 3600 else None,
                         "kernel": "insert (PNN)",
                         "algorithmic_bytes": ins_bytes, "peak_kind": peak_kind},
            "issue_roofline": issue,
            "stage_rooflines": {
                "fill_and_clear": {"algorithmic_bytes": fill_bytes,
                                   "achieved_gbs": fill_bytes / (fill_ms / 1e3) / 1e9,
                                   "frac": fill_bytes / (fill_ms / 1e3) / 1e9 / peak,
                                   "clear_bytes": clear_bytes,
                                   "raw_gbs_with_clear": (fill_bytes + clear_bytes) /
                                                         (fill_ms / 1e3) / 1e9},
                "project": {"algorithmic_bytes": proj_bytes,
                            "achieved_gbs": proj_bytes / (proj_ms / 1e3) / 1e9,
                            "frac": proj_bytes / (proj_ms / 1e3) / 1e9 / peak}},
            "pipeline_roofline": {"algorithmic_bytes_per_step": step_bytes,
                                  "achieved_gbs": step_bytes / (ms_per_step / 1e3) / 1e9,
                                  "frac": step_bytes / (ms_per_step / 1e3) / 1e9 / peak,
                                  "bytes": "insert (frames + 16 B per touched voxel) + fill "
                                           "(8 + 1 + 1/8 B per voxel) + projection; the "
                                           "zeros the fill writes for the next sweep are "
                                           "not counted",
                                  "clear_bytes_per_step": clear_bytes},
            "touched_voxels": touched, "pixel_hits": hits,
            "p50_frame_to_render_ms": streaming["p50_ms"] if streaming else None,
            "p99_frame_to_render_ms": streaming["p99_ms"] if streaming else None,
            "streaming": streaming,
            "variants": variants,
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches_per_step * K,
            "autotune": tune, "cuda_graph": graph, "batches_of_30": b30,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
